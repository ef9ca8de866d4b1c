// FP32 SIMT GEMM for the predictor's projections:  C[M][N] = epi(A[M][K] . Wt[K][N]).
//
// A is an activation matrix (one row per (stream, step)), Wt a weight matrix
// stored K-major ([in][out], the transpose of nn.Linear's [out][in]).
//
// Determinism contract: every output element is the chain
//     acc = 0; for k = 0..K-1: acc = fma(A[m][k], Wt[k][n], acc)
// followed by the epilogue, whatever the tile shape or the row's position in
// the batch.  The compression path (rows = streams x time chunk) and the
// decompression path (rows = streams, one step) therefore produce
// bit-identical logits for the same stream history, which keeps the range
// coders of both sides in lockstep (paper, "Determinism and synchronisation").
#pragma once
#include "common.cuh"

namespace boa {

enum Epi : int {
    kEpiStore = 0,      // C = acc
    kEpiBias = 1,       // C = acc + b[n]
    kEpiResid = 2,      // C = C + acc                 (residual add in place)
    kEpiBiasGelu = 3,   // C = gelu(acc + b[n])
    kEpiBiasResid = 4,  // C = C + (acc + b[n])
};

constexpr int kGemmThreads = 256;
constexpr int kGemmBK = 8;

// BM x BN tile, 16 x 16 threads, each thread a TM x TN micro-tile split in
// groups of 4 rows / columns spaced BM/2 (BN/2) apart so the shared-memory
// float4 reads of a warp are conflict-free.
template <int BM, int BN, int EPI>
__global__ void __launch_bounds__(kGemmThreads)
k_gemm_fp32(const float* __restrict__ A, const float* __restrict__ Wt, const float* __restrict__ bias,
            float* __restrict__ Cm, int M, int N, int K) {
    pdl_launch_next();
    pdl_wait_prev();
    constexpr int TM = BM / 16, TN = BN / 16;
    constexpr int GM = TM / 4, GN = TN / 4;           // groups of 4
    constexpr int A_F4 = BM * kGemmBK / 4;            // float4 per A tile
    constexpr int B_F4 = BN * kGemmBK / 4;
    constexpr int A_PER = (A_F4 + kGemmThreads - 1) / kGemmThreads;
    constexpr int B_PER = (B_F4 + kGemmThreads - 1) / kGemmThreads;
    static_assert(TM % 4 == 0 && TN % 4 == 0, "micro-tile must be a multiple of 4");

    __shared__ __align__(16) float As[2][kGemmBK][BM];
    __shared__ __align__(16) float Bs[2][kGemmBK][BN];

    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

    float4 ra[A_PER], rb[B_PER];

    auto load_tiles = [&](int k0) {
#pragma unroll
        for (int p = 0; p < A_PER; p++) {
            int i = tid + p * kGemmThreads;
            ra[p] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < A_F4) {
                int row = i / (kGemmBK / 4), kq = (i % (kGemmBK / 4)) * 4;
                if (m0 + row < M) ra[p] = *reinterpret_cast<const float4*>(A + (size_t)(m0 + row) * K + k0 + kq);
            }
        }
#pragma unroll
        for (int p = 0; p < B_PER; p++) {
            int i = tid + p * kGemmThreads;
            rb[p] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < B_F4) {
                int kr = i / (BN / 4), nq = (i % (BN / 4)) * 4;
                if (n0 + nq < N) rb[p] = *reinterpret_cast<const float4*>(Wt + (size_t)(k0 + kr) * N + n0 + nq);
            }
        }
    };
    auto store_tiles = [&](int buf) {
#pragma unroll
        for (int p = 0; p < A_PER; p++) {
            int i = tid + p * kGemmThreads;
            if (i < A_F4) {
                int row = i / (kGemmBK / 4), kq = (i % (kGemmBK / 4)) * 4;
                As[buf][kq + 0][row] = ra[p].x;
                As[buf][kq + 1][row] = ra[p].y;
                As[buf][kq + 2][row] = ra[p].z;
                As[buf][kq + 3][row] = ra[p].w;
            }
        }
#pragma unroll
        for (int p = 0; p < B_PER; p++) {
            int i = tid + p * kGemmThreads;
            if (i < B_F4) {
                int kr = i / (BN / 4), nq = (i % (BN / 4)) * 4;
                *reinterpret_cast<float4*>(&Bs[buf][kr][nq]) = rb[p];
            }
        }
    };

    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) acc[i][j] = 0.0f;

    const int nk = K / kGemmBK;
    load_tiles(0);
    store_tiles(0);
    __syncthreads();
    for (int kt = 0; kt < nk; kt++) {
        const int cur = kt & 1;
        if (kt + 1 < nk) load_tiles((kt + 1) * kGemmBK);
#pragma unroll
        for (int kk = 0; kk < kGemmBK; kk++) {
            float a[TM], b[TN];
#pragma unroll
            for (int g = 0; g < GM; g++) {
                float4 v = *reinterpret_cast<const float4*>(&As[cur][kk][g * (BM / GM) + ty * 4]);
                a[g * 4 + 0] = v.x; a[g * 4 + 1] = v.y; a[g * 4 + 2] = v.z; a[g * 4 + 3] = v.w;
            }
#pragma unroll
            for (int g = 0; g < GN; g++) {
                float4 v = *reinterpret_cast<const float4*>(&Bs[cur][kk][g * (BN / GN) + tx * 4]);
                b[g * 4 + 0] = v.x; b[g * 4 + 1] = v.y; b[g * 4 + 2] = v.z; b[g * 4 + 3] = v.w;
            }
#pragma unroll
            for (int i = 0; i < TM; i++)
#pragma unroll
                for (int j = 0; j < TN; j++) acc[i][j] = __fmaf_rn(a[i], b[j], acc[i][j]);
        }
        if (kt + 1 < nk) store_tiles(cur ^ 1);
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < TM; i++) {
        const int m = m0 + (i / 4) * (BM / GM) + ty * 4 + (i % 4);
        if (m >= M) continue;
#pragma unroll
        for (int g = 0; g < GN; g++) {
            const int n = n0 + g * (BN / GN) + tx * 4;
            if (n >= N) continue;   // N % 4 == 0, so a group is all in or all out
            float* cp = Cm + (size_t)m * N + n;
            float4 o;
            float* ov = reinterpret_cast<float*>(&o);
            float4 old = make_float4(0.f, 0.f, 0.f, 0.f);
            if (EPI == kEpiResid || EPI == kEpiBiasResid) old = *reinterpret_cast<const float4*>(cp);
            const float* oldv = reinterpret_cast<const float*>(&old);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                float v = acc[i][g * 4 + q];
                if (EPI == kEpiBias || EPI == kEpiBiasGelu || EPI == kEpiBiasResid) v = __fadd_rn(v, bias[n + q]);
                if (EPI == kEpiBiasGelu) v = gelu_f(v);
                if (EPI == kEpiResid || EPI == kEpiBiasResid) v = __fadd_rn(oldv[q], v);
                ov[q] = v;
            }
            *reinterpret_cast<float4*>(cp) = o;
        }
    }
}

}  // namespace boa
