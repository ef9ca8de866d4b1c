// Selective scan for training (paper App. A recurrence; reverse-mode
// gradient): forward over whole sequences keeping only the state entering
// every chunk, and a backward that recomputes each chunk's states from that
// entry state (latest chunk first) and runs the reverse recurrence
//     g_t = C_t dy_t + a_{t+1} g_{t+1},   a_t = exp(delta_t A).
// Layouts: u, delta, y, du, ddelta [Bsz][T][E]; Bm, Cm [Bsz][T][N];
// A [E][N]; D [E]; hin [Bsz][nchunk][N][E]; scratch hs [Bsz][chunk][N][E].
// dB / dC are summed over each CTA's 128 channels into per-block partials
// [Bsz][T][E/128][N]; dA / dD are per-sequence partials [Bsz][E][N], [Bsz][E]
// (the caller sums the partials, so no atomics are involved).
#pragma once
#include "common.cuh"

namespace boa {

constexpr int kTrainThreads = 128;

template <int NS>
__global__ void __launch_bounds__(kTrainThreads)
k_scan_train_fwd(int T, int E, int chunk, const float* __restrict__ u, const float* __restrict__ delta,
                 const float* __restrict__ A, const float* __restrict__ Bm, const float* __restrict__ Cm,
                 const float* __restrict__ D, float* __restrict__ y, float* __restrict__ hin) {
    const int b = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= E) return;
    const int nck = (T + chunk - 1) / chunk;
    float a[NS], h[NS];
#pragma unroll
    for (int n = 0; n < NS; n++) { a[n] = A[(size_t)c * NS + n]; h[n] = 0.f; }
    const float dv = D[c];
    for (int t = 0; t < T; t++) {
        if (t % chunk == 0) {
            const int k = t / chunk;
#pragma unroll
            for (int n = 0; n < NS; n++) hin[(((size_t)b * nck + k) * NS + n) * E + c] = h[n];
        }
        const size_t r = (size_t)b * T + t;
        const float dl = delta[r * E + c], uc = u[r * E + c];
        const float du = dl * uc;
        float acc = 0.f;
#pragma unroll
        for (int n = 0; n < NS; n++) {
            h[n] = __expf(dl * a[n]) * h[n] + du * Bm[r * NS + n];
            acc += Cm[r * NS + n] * h[n];
        }
        y[r * E + c] = acc + dv * uc;
    }
}

template <int NS>
__global__ void __launch_bounds__(kTrainThreads)
k_scan_train_bwd(int T, int E, int chunk, const float* __restrict__ u, const float* __restrict__ delta,
                 const float* __restrict__ A, const float* __restrict__ Bm, const float* __restrict__ Cm,
                 const float* __restrict__ D, const float* __restrict__ dy, const float* __restrict__ hin,
                 float* __restrict__ hs, float* __restrict__ du, float* __restrict__ ddelta,
                 float* __restrict__ dA_part, float* __restrict__ dD_part, float* __restrict__ dB_part,
                 float* __restrict__ dC_part) {
    __shared__ float red[kTrainThreads / 32][2 * NS];
    const int b = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nblk = gridDim.x;
    const bool live = c < E;
    const int nck = (T + chunk - 1) / chunk;
    float a[NS], g[NS], dA[NS];
#pragma unroll
    for (int n = 0; n < NS; n++) { a[n] = live ? A[(size_t)c * NS + n] : 0.f; g[n] = 0.f; dA[n] = 0.f; }
    const float dv = live ? D[c] : 0.f;
    float dD = 0.f;
    for (int k = nck - 1; k >= 0; k--) {
        const int t0 = k * chunk, t1 = min(T, t0 + chunk);
        // recompute the chunk's states from its entry state
        if (live) {
            float h[NS];
#pragma unroll
            for (int n = 0; n < NS; n++) h[n] = hin[(((size_t)b * nck + k) * NS + n) * E + c];
            for (int t = t0; t < t1; t++) {
                const size_t r = (size_t)b * T + t;
                const float dl = delta[r * E + c], uc = u[r * E + c];
                const float dub = dl * uc;
#pragma unroll
                for (int n = 0; n < NS; n++) {
                    h[n] = __expf(dl * a[n]) * h[n] + dub * Bm[r * NS + n];
                    hs[(((size_t)b * chunk + (t - t0)) * NS + n) * E + c] = h[n];
                }
            }
        }
        // reverse recurrence over the chunk
        for (int t = t1 - 1; t >= t0; t--) {
            const size_t r = (size_t)b * T + t;
            float pB[NS], pC[NS];
            if (live) {
                const float dl = delta[r * E + c], uc = u[r * E + c], gy = dy[r * E + c];
                float dd = 0.f, duc = 0.f;
#pragma unroll
                for (int n = 0; n < NS; n++) {
                    const float ht = hs[(((size_t)b * chunk + (t - t0)) * NS + n) * E + c];
                    const float hp = t > t0 ? hs[(((size_t)b * chunk + (t - 1 - t0)) * NS + n) * E + c]
                                            : hin[(((size_t)b * nck + k) * NS + n) * E + c];
                    const float Bn = Bm[r * NS + n], Cn = Cm[r * NS + n];
                    const float an = __expf(dl * a[n]);
                    g[n] += gy * Cn;
                    pC[n] = gy * ht;
                    const float da = g[n] * hp;
                    dd += da * an * a[n] + g[n] * Bn * uc;
                    dA[n] += da * an * dl;
                    pB[n] = g[n] * dl * uc;
                    duc += g[n] * dl * Bn;
                    g[n] *= an;
                }
                duc += gy * dv;
                dD += gy * uc;
                du[r * E + c] = duc;
                ddelta[r * E + c] = dd;
            } else {
#pragma unroll
                for (int n = 0; n < NS; n++) { pB[n] = 0.f; pC[n] = 0.f; }
            }
            // sum pB, pC over the CTA's channels (fixed butterfly, then warps in order)
#pragma unroll
            for (int n = 0; n < NS; n++) {
                float vb = pB[n], vc = pC[n];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    vb += __shfl_xor_sync(0xffffffffu, vb, o);
                    vc += __shfl_xor_sync(0xffffffffu, vc, o);
                }
                if (lane == 0) { red[warp][n] = vb; red[warp][NS + n] = vc; }
            }
            __syncthreads();
            if (threadIdx.x < 2 * NS) {
                float s = 0.f;
                for (int w = 0; w < kTrainThreads / 32; w++) s += red[w][threadIdx.x];
                const size_t o = ((size_t)r * nblk + blockIdx.x) * NS;
                if (threadIdx.x < NS) dB_part[o + threadIdx.x] = s;
                else dC_part[o + threadIdx.x - NS] = s;
            }
            __syncthreads();
        }
    }
    if (live) {
#pragma unroll
        for (int n = 0; n < NS; n++) dA_part[((size_t)b * E + c) * NS + n] = dA[n];
        dD_part[(size_t)b * E + c] = dD;
    }
}

}  // namespace boa
