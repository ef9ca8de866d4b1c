// Kernels of the native training step (boa_train_step): the predictor's
// forward over (sequence x position) rows keeping what the backward needs,
// the reverse-mode gradient of the mean base-256 cross-entropy (paper,
// "Entropy-Based Compression and Cross-Entropy Loss"), and AdamW.
//
// Everything is FP32 on the CUDA cores, in a fixed order: a row-parallel
// kernel owns its rows outright, and every sum over rows (weight gradients,
// bias and norm gradients, the loss) is taken per chunk of rows into partial
// arrays that a second kernel adds in chunk order, so a step gives the same
// bits every time (no atomics).  The selective scan's own forward and
// backward are k_scan_train_fwd / k_scan_train_bwd (scan_train.cuh).
//
// Row r of a batch of sequences of T predicted positions is (b, t) =
// (r / T, r % T); its input byte is tok[b * seqlen + t], its target byte
// tok[b * seqlen + t + 1] (seqlen = T + 1).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace boa {

constexpr int kTrBlock = 256;

// x[r][:] = embed[tok(r)][:]
__global__ void k_tr_embed(const uint8_t* __restrict__ tok, int T, int seqlen, const float* __restrict__ embed,
                           float* __restrict__ x, long long rows, int d) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * d) return;
    const long long r = i / d;
    const int j = (int)(i % d);
    const int v = tok[(r / T) * seqlen + r % T];
    x[i] = embed[(size_t)v * d + j];
}

// LayerNorm over rows of d <= 256 (one warp per row, d a multiple of 32):
// y = (x - mean) * rstd * g + b with rstd = 1 / sqrt(var + 1e-5).
__global__ void k_tr_ln_fwd(const float* __restrict__ x, const float* __restrict__ g, const float* __restrict__ b,
                            float* __restrict__ y, float* __restrict__ mean, float* __restrict__ rstd, long long rows,
                            int d) {
    const int lane = threadIdx.x & 31;
    const long long r = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (r >= rows) return;
    const int vpt = d / 32;
    float v[8];
    float s = 0.f;
    for (int i = 0; i < vpt; i++) {
        v[i] = x[r * d + lane + 32 * i];
        s += v[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float mu = s / d;
    float q = 0.f;
    for (int i = 0; i < vpt; i++) {
        const float c = v[i] - mu;
        q += c * c;
    }
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    const float rs = 1.0f / sqrtf(q / d + 1e-5f);
    for (int i = 0; i < vpt; i++) {
        const int j = lane + 32 * i;
        y[r * d + j] = (v[i] - mu) * rs * g[j] + b[j];
    }
    if (lane == 0) {
        mean[r] = mu;
        rstd[r] = rs;
    }
}

// LayerNorm backward: with xh = (x - mean) rstd and gy = dy * g,
//   dx = rstd (gy - mean(gy) - xh mean(gy xh))   (added to dx when accumulate)
// and dyxh = dy * xh, whose column sums give the gain gradient.
__global__ void k_tr_ln_bwd(const float* __restrict__ dy, const float* __restrict__ x, const float* __restrict__ mean,
                            const float* __restrict__ rstd, const float* __restrict__ g, float* __restrict__ dx,
                            float* __restrict__ dyxh, long long rows, int d, int accumulate) {
    const int lane = threadIdx.x & 31;
    const long long r = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (r >= rows) return;
    const int vpt = d / 32;
    const float mu = mean[r], rs = rstd[r];
    float xh[8], gy[8];
    float s1 = 0.f, s2 = 0.f;
    for (int i = 0; i < vpt; i++) {
        const int j = lane + 32 * i;
        const float dyv = dy[r * d + j];
        xh[i] = (x[r * d + j] - mu) * rs;
        gy[i] = dyv * g[j];
        dyxh[r * d + j] = dyv * xh[i];
        s1 += gy[i];
        s2 += gy[i] * xh[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const float m1 = s1 / d, m2 = s2 / d;
    for (int i = 0; i < vpt; i++) {
        const int j = lane + 32 * i;
        const float v = rs * (gy[i] - m1 - xh[i] * m2);
        dx[r * d + j] = accumulate ? dx[r * d + j] + v : v;
    }
}

// C[M][N] (+)= A[M][K] . B[K][N] (+ bias[N]); row-major with leading
// dimensions; 64 x 64 tiles, 16 x 16 threads of 4 x 4 outputs, K in steps of
// 16; every output is a sequential sum over k.
constexpr int kTrTile = 64, kTrTk = 16;

__global__ void __launch_bounds__(256)
k_tr_gemm_nn(int M, int N, int K, const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
             float* __restrict__ C, int ldc, const float* __restrict__ bias, int accumulate) {
    __shared__ float sA[kTrTk][kTrTile + 4];
    __shared__ float sB[kTrTk][kTrTile + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * kTrTile, n0 = blockIdx.x * kTrTile;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kTrTk) {
        for (int i = threadIdx.x; i < kTrTk * kTrTile; i += 256) {
            const int mm = i / kTrTk, kk = i % kTrTk;      // A tile: 64 rows x 16 k
            const int gm = m0 + mm, gk = k0 + kk;
            sA[kk][mm] = (gm < M && gk < K) ? A[(size_t)gm * lda + gk] : 0.f;
            const int kb = i / kTrTile, nb = i % kTrTile;  // B tile: 16 k x 64 cols
            const int gkb = k0 + kb, gn = n0 + nb;
            sB[kb][nb] = (gkb < K && gn < N) ? B[(size_t)gkb * ldb + gn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTrTk; kk++) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                a[i] = sA[kk][ty + 16 * i];
                b[i] = sB[kk][tx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = __fmaf_rn(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            float v = acc[i][j];
            if (bias) v += bias[gn];
            float* cp = C + (size_t)gm * ldc + gn;
            *cp = accumulate ? *cp + v : v;
        }
    }
}

// part[z][N][K] = sum over rows r of chunk z of A[r][n] B[r][k]  (A: rows x
// N with leading dimension lda, B: rows x K with ldb); chunk z covers rows
// [z * rpp, min(R, (z + 1) * rpp)).
__global__ void __launch_bounds__(256)
k_tr_gemm_tn(long long R, int N, int K, const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
             float* __restrict__ part, long long rpp) {
    __shared__ float sA[kTrTk][kTrTile + 4];
    __shared__ float sB[kTrTk][kTrTile + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int n0 = blockIdx.y * kTrTile, k0 = blockIdx.x * kTrTile;
    const long long r_beg = (long long)blockIdx.z * rpp, r_end = min(R, r_beg + rpp);
    float acc[4][4] = {};
    for (long long r0 = r_beg; r0 < r_end; r0 += kTrTk) {
        for (int i = threadIdx.x; i < kTrTk * kTrTile; i += 256) {
            const int rr = i / kTrTile, cc = i % kTrTile;
            const long long gr = r0 + rr;
            sA[rr][cc] = (gr < r_end && n0 + cc < N) ? A[(size_t)gr * lda + n0 + cc] : 0.f;
            sB[rr][cc] = (gr < r_end && k0 + cc < K) ? B[(size_t)gr * ldb + k0 + cc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < kTrTk; rr++) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                a[i] = sA[rr][ty + 16 * i];
                b[i] = sB[rr][tx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = __fmaf_rn(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* out = part + (size_t)blockIdx.z * N * K;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int n = n0 + ty + 16 * i;
        if (n >= N) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int k = k0 + tx + 16 * j;
            if (k < K) out[(size_t)n * K + k] = acc[i][j];
        }
    }
}

// part[z][j] = sum over rows of chunk z of A[r][j]  (j < n)
__global__ void k_tr_colsum(const float* __restrict__ A, long long R, int n, int lda, float* __restrict__ part,
                            long long rpp) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const long long r_beg = (long long)blockIdx.y * rpp, r_end = min(R, r_beg + rpp);
    float s = 0.f;
    for (long long r = r_beg; r < r_end; r++) s += A[(size_t)r * lda + j];
    part[(size_t)blockIdx.y * n + j] = s;
}

// out[i] (+)= sum_{z < P} part[z][i], in order of z; then * scale[i] when given.
__global__ void k_tr_reduce(const float* __restrict__ part, int P, size_t count, float* __restrict__ out,
                            int accumulate, const float* __restrict__ scale) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float s = 0.f;
    for (int z = 0; z < P; z++) s += part[(size_t)z * count + i];
    if (scale) s *= scale[i];
    out[i] = accumulate ? out[i] + s : s;
}

// Causal depthwise conv + SiLU over whole sequences (window zero at t = 0):
// cpre[t] = b + sum_k w[c][k] xi[t - K + 1 + k], u = SiLU(cpre); w in the
// weight file's [E][K] layout, xi the first E columns of xz (row stride 2E).
__global__ void k_tr_conv_fwd(const float* __restrict__ xz, int E, const float* __restrict__ w,
                              const float* __restrict__ b, float* __restrict__ cpre, float* __restrict__ u, int T,
                              int K) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= E) return;
    const size_t r0 = (size_t)blockIdx.y * T;
    float wk[4], win[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < K; k++) wk[k] = w[(size_t)c * K + k];
    const float bc = b[c];
    for (int t = 0; t < T; t++) {
        const size_t r = r0 + t;
        const float xi = xz[r * 2 * E + c];
        float acc = bc;
        for (int k = 0; k < K - 1; k++) acc += wk[k] * win[k];
        acc += wk[K - 1] * xi;
        for (int k = 0; k + 1 < K - 1; k++) win[k] = win[k + 1];
        if (K > 1) win[K - 2] = xi;
        cpre[r * E + c] = acc;
        u[r * E + c] = acc / (1.0f + expf(-acc));
    }
}

// dxi[t] = sum_k w[c][k] dcpre[t + K - 1 - k] (within the sequence), written
// into the first E columns of dxz (row stride 2E).
__global__ void k_tr_conv_bwd(const float* __restrict__ dcpre, const float* __restrict__ w, float* __restrict__ dxz,
                              int T, int E, int K) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= E) return;
    const size_t r0 = (size_t)blockIdx.y * T;
    float wk[4];
    for (int k = 0; k < K; k++) wk[k] = w[(size_t)c * K + k];
    for (int t = 0; t < T; t++) {
        float s = 0.f;
        for (int k = 0; k < K; k++) {
            const int tt = t + K - 1 - k;
            if (tt < T) s += wk[k] * dcpre[(r0 + tt) * E + c];
        }
        dxz[(r0 + t) * 2 * E + c] = s;
    }
}

// Conv weight and bias gradients over a chunk of rows: part[z][c][k] (k < K)
// = sum_r dcpre[r][c] xi[r - K + 1 + k][c] (same sequence), part[z][c][K] =
// sum_r dcpre[r][c].
__global__ void k_tr_conv_wgrad(const float* __restrict__ dcpre, const float* __restrict__ xz, float* __restrict__ part,
                                int T, int E, int K, long long R, long long rpp) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= E) return;
    const long long r_beg = (long long)blockIdx.y * rpp, r_end = min(R, r_beg + rpp);
    float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (long long r = r_beg; r < r_end; r++) {
        const float g = dcpre[(size_t)r * E + c];
        const int t = (int)(r % T);
        for (int k = 0; k < K; k++) {
            const int back = K - 1 - k;
            if (t >= back) s[k] += g * xz[(size_t)(r - back) * 2 * E + c];
        }
        s[K] += g;
    }
    float* out = part + (size_t)blockIdx.y * E * (K + 1) + (size_t)c * (K + 1);
    for (int k = 0; k <= K; k++) out[k] = s[k];
}

// BF16 operands of the tensor-core projections in a BF16 model's training
// step (FP32 master weights; FP32 accumulation in the GEMMs).
//
// dst[i] = bf16(src[i]), round to nearest even.
__global__ void k_tr_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// Transposed copy: dst[c][r] = bf16(src[r][c]) for r < R, c < C (src has
// leading dimension lds); dst rows hold Rp >= R entries, zero from R on.
// 32 x 32 tiles through shared memory, so both sides are coalesced; block
// (32, 8), grid (Rp / 32, ceil(C / 32)).
__global__ void k_tr_bf16_t(const float* __restrict__ src, int lds, long long R, int C, long long Rp,
                            __nv_bfloat16* __restrict__ dst) {
    __shared__ float tile[32][33];
    const long long r0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const long long r = r0 + i;
        const int c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < R && c < C) ? src[r * lds + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int c = c0 + i;
        const long long r = r0 + threadIdx.x;
        if (c < C && r < Rp) dst[(size_t)c * Rp + r] = __float2bfloat16_rn(tile[threadIdx.x][i]);
    }
}

// Elementwise pieces.
__global__ void k_tr_softplus(const float* __restrict__ pre, float* __restrict__ out, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = pre[i];
    out[i] = v > 20.f ? v : log1pf(expf(v));
}

__global__ void k_tr_softplus_bwd(const float* __restrict__ dout, const float* __restrict__ pre, float* __restrict__ dpre,
                                  size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = pre[i];
    dpre[i] = v > 20.f ? dout[i] : dout[i] / (1.0f + expf(-v));
}

__global__ void k_tr_neg_exp(const float* __restrict__ a_log, float* __restrict__ a, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = -expf(a_log[i]);
}

// dbc rows [delta (r) | B (N) | C (N)] -> B, C [rows][N]
__global__ void k_tr_split_bc(const float* __restrict__ dbc, int r, int N, float* __restrict__ Bm, float* __restrict__ Cm,
                              long long rows) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * N) return;
    const long long row = i / N;
    const int n = (int)(i % N);
    const float* src = dbc + (size_t)row * (r + 2 * N);
    Bm[i] = src[r + n];
    Cm[i] = src[r + N + n];
}

// yg = ys * SiLU(z), z the last E columns of xz
__global__ void k_tr_gate_fwd(const float* __restrict__ ys, const float* __restrict__ xz, int E, float* __restrict__ yg,
                              long long rows) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * E) return;
    const long long row = i / E;
    const float z = xz[(size_t)row * 2 * E + E + i % E];
    yg[i] = ys[i] * (z / (1.0f + expf(-z)));
}

// dys = dyg SiLU(z); dz = dyg ys SiLU'(z) with SiLU'(z) = s (1 + z (1 - s)), s = sigmoid(z)
__global__ void k_tr_gate_bwd(const float* __restrict__ dyg, const float* __restrict__ ys, const float* __restrict__ xz,
                              int E, float* __restrict__ dys, float* __restrict__ dxz, long long rows) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * E) return;
    const long long row = i / E;
    const int c = (int)(i % E);
    const float z = xz[(size_t)row * 2 * E + E + c];
    const float s = 1.0f / (1.0f + expf(-z));
    dys[i] = dyg[i] * z * s;
    dxz[(size_t)row * 2 * E + E + c] = dyg[i] * ys[i] * s * (1.0f + z * (1.0f - s));
}

// dcpre = du SiLU'(cpre)
__global__ void k_tr_silu_bwd(const float* __restrict__ du, const float* __restrict__ cpre, float* __restrict__ dcpre,
                              size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = cpre[i];
    const float s = 1.0f / (1.0f + expf(-v));
    dcpre[i] = du[i] * s * (1.0f + v * (1.0f - s));
}

// dbc gradient rows: [d_delta (r) | sum_blk dB | sum_blk dC] (blocks in order)
__global__ void k_tr_assemble_ddbc(const float* __restrict__ ddl, const float* __restrict__ dB_part,
                                   const float* __restrict__ dC_part, int nblk, int r, int N, float* __restrict__ ddbc,
                                   long long rows) {
    const int W = r + 2 * N;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * W) return;
    const long long row = i / W;
    const int j = (int)(i % W);
    float v;
    if (j < r) {
        v = ddl[(size_t)row * r + j];
    } else {
        const bool isB = j < r + N;
        const int n = isB ? j - r : j - r - N;
        const float* p = (isB ? dB_part : dC_part) + (size_t)row * nblk * N + n;
        v = 0.f;
        for (int b = 0; b < nblk; b++) v += p[(size_t)b * N];
    }
    ddbc[i] = v;
}

// Loss and logit gradient, one warp per row: loss_row = logsumexp(l) - l[y]
// (natural log), dl = (softmax(l) - onehot(y)) * scale.
__global__ void k_tr_xent(const float* __restrict__ logits, const uint8_t* __restrict__ tok, int T, int seqlen,
                          float* __restrict__ dlogits, float* __restrict__ loss_rows, long long rows, float scale) {
    const int lane = threadIdx.x & 31;
    const long long r = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (r >= rows) return;
    const int y = tok[(r / T) * seqlen + r % T + 1];
    const float* l = logits + (size_t)r * 256;
    float v[8];
    float mx = -INFINITY;
    for (int i = 0; i < 8; i++) {
        v[i] = l[lane + 32 * i];
        mx = fmaxf(mx, v[i]);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float s = 0.f;
    for (int i = 0; i < 8; i++) {
        v[i] = expf(v[i] - mx);
        s += v[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    for (int i = 0; i < 8; i++) {
        const int j = lane + 32 * i;
        dlogits[(size_t)r * 256 + j] = (v[i] / s - (j == y ? 1.f : 0.f)) * scale;
    }
    if (lane == 0) loss_rows[r] = mx + logf(s) - l[y];
}

// out[0] = sum of v[0..n) (one CTA of kTrBlock threads: strided partials in
// thread order, then a fixed tree).
__global__ void k_tr_sum(const float* __restrict__ v, long long n, float* __restrict__ out) {
    __shared__ float red[kTrBlock];
    float s = 0.f;
    for (long long i = threadIdx.x; i < n; i += kTrBlock) s += v[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kTrBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// Embedding gradient: one CTA per byte value v, thread j sums dx[r][j] over
// the rows whose input byte is v, in row order.
__global__ void k_tr_embed_bwd(const float* __restrict__ dx, const uint8_t* __restrict__ tok, int T, int seqlen,
                               long long rows, int d, float* __restrict__ g) {
    const int v = blockIdx.x;
    const int j = threadIdx.x;
    if (j >= d) return;
    float s = 0.f;
    for (long long r = 0; r < rows; r++)
        if (tok[(r / T) * seqlen + r % T] == v) s += dx[(size_t)r * d + j];
    g[(size_t)v * d + j] = s;
}

// AdamW (decoupled weight decay): p -= lr (wd p + mhat / (sqrt(vhat) + eps)).
__global__ void k_tr_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                           float* __restrict__ m2, size_t n, float lr, float b1, float b2, float eps, float wd,
                           float bc1, float bc2) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float pi = p[i] * (1.f - lr * wd);
    p[i] = pi - lr * (a / bc1) / (sqrtf(b / bc2) + eps);
}

}  // namespace boa
