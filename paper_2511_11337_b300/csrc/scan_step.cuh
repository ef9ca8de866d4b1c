// Decode-step selective scan (one step of every stream, Eq. 2 of the SSM
// recurrence), persistent and fed by bulk copies.
//
// In decompression every step reads and rewrites each stream's whole SSM
// state (N x E floats, 32 KB at E = 512), so the kernel is bound by HBM
// traffic and needs many bytes in flight per SM.  Each CTA walks the streams
// s = blockIdx.x, blockIdx.x + gridDim.x, ...; thread 0 keeps `stages` of
// them in flight in a shared-memory ring (the stream's state [N][E], its u
// and z rows and its dbc row, one cp.async.bulk each, completing on one
// mbarrier per stage).  Every thread owns two adjacent channels, and their
// A2t and W_dt columns stay in registers for the kernel's lifetime.  New
// states go from registers straight to hstate with coalesced 8-byte stores.
//
// Per channel the arithmetic is exactly that of k_scan (same operations,
// same order), so a stream decoded here sees the same rows as when it was
// encoded.
//
// Waits are bounded (about 2 s of globaltimer).  On expiry the CTA records
// code 3 in *err, waits (bounded again) for the copies it has in flight and
// returns.
#pragma once
#include "gemm_tc.cuh"
#include "kernels.cuh"

namespace boa {

// 1-D bulk copy global -> shared, completing on an mbarrier (both addresses
// 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"((uint64_t)__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

constexpr int kStepMaxStages = 4;

// Floats per ring stage: state, u row, z row, dbc row.
__host__ __device__ constexpr int step_stage_floats(int NS, int R, int E) { return NS * E + 2 * E + R + 2 * NS; }

template <int NS, int R>
__global__ void __launch_bounds__(512)
k_scan_step_bulk(const float* __restrict__ u, const float* __restrict__ xz, const float* __restrict__ dbc,
                 const float* __restrict__ dtwt, const float* __restrict__ dt_b, const float* __restrict__ A2t,
                 const float* __restrict__ Dv, float* __restrict__ hstate, float* __restrict__ yg,
                 __nv_bfloat16* __restrict__ yg_b, int E, int S, int stages, int* __restrict__ err, F8Out f8) {
    constexpr int W = R + 2 * NS;
    static_assert(W % 4 == 0, "the dbc row is copied in 16-byte units");
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[kStepMaxStages];
    __shared__ float red[2][16];                 // FP8 form: per-warp row maxima (up to 16 warps)
    const int sf = step_stage_floats(NS, R, E);
    float* ring = reinterpret_cast<float*>(smem_raw);
    const int tid = threadIdx.x;
    const int c = 2 * tid;                       // blockDim.x == E / 2
    const int G = gridDim.x;
    const int mine = (int)blockIdx.x < S ? (S - 1 - (int)blockIdx.x) / G + 1 : 0;

    auto issue = [&](int k) {                    // k-th stream of this CTA into stage k % stages
        const int s = blockIdx.x + k * G;
        float* st = ring + (size_t)(k % stages) * sf;
        uint64_t* bar = &full[k % stages];
        mbar_expect_tx(bar, (uint32_t)sf * 4u);
        bulk_g2s(st, hstate + (size_t)s * NS * E, (uint32_t)(NS * E * 4), bar);
        bulk_g2s(st + NS * E, u + (size_t)s * E, (uint32_t)(E * 4), bar);
        bulk_g2s(st + NS * E + E, xz + (size_t)s * 2 * E + E, (uint32_t)(E * 4), bar);
        bulk_g2s(st + NS * E + 2 * E, dbc + (size_t)s * W, (uint32_t)(W * 4), bar);
    };

    int issued = 0;
    pdl_launch_next();
    if (tid == 0) {
        for (int i = 0; i < stages; i++) mbar_init(&full[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    pdl_wait_prev();                             // u, z, dbc and the state come from earlier kernels
    if (tid == 0)
        for (; issued < min(stages, mine); issued++) issue(issued);

    float a2[NS][2], wdt[R][2];
#pragma unroll
    for (int n = 0; n < NS; n++) {
        const float2 v = *reinterpret_cast<const float2*>(A2t + (size_t)n * E + c);
        a2[n][0] = v.x;
        a2[n][1] = v.y;
    }
#pragma unroll
    for (int j = 0; j < R; j++) {
        const float2 v = *reinterpret_cast<const float2*>(dtwt + (size_t)j * E + c);
        wdt[j][0] = v.x;
        wdt[j][1] = v.y;
    }
    const float2 bdt = *reinterpret_cast<const float2*>(dt_b + c);
    const float2 dv = *reinterpret_cast<const float2*>(Dv + c);

    int k = 0;
    bool aborted = false;
    for (; k < mine; k++) {
        const bool ok = mbar_wait(&full[k % stages], (uint32_t)((k / stages) & 1));
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        const int s = blockIdx.x + k * G;
        const float* hb = ring + (size_t)(k % stages) * sf;
        const float* ub = hb + NS * E;
        const float* zb = ub + E;
        const float* db = zb + E;
        const float2 u2 = *reinterpret_cast<const float2*>(ub + c);
        const float2 z2 = *reinterpret_cast<const float2*>(zb + c);
        float pre0 = 0.f, pre1 = 0.f;
#pragma unroll
        for (int j = 0; j < R; j++) {
            const float dj = db[j];
            pre0 = __fmaf_rn(wdt[j][0], dj, pre0);
            pre1 = __fmaf_rn(wdt[j][1], dj, pre1);
        }
        const float delta0 = softplus_f(__fadd_rn(pre0, bdt.x));
        const float delta1 = softplus_f(__fadd_rn(pre1, bdt.y));
        const float du0 = __fmul_rn(delta0, u2.x);
        const float du1 = __fmul_rn(delta1, u2.y);
        float y0 = 0.f, y1 = 0.f;
        float* hout = hstate + (size_t)s * NS * E + c;
#pragma unroll
        for (int n = 0; n < NS; n++) {
            const float2 h2 = *reinterpret_cast<const float2*>(hb + n * E + c);
            const float Bn = db[R + n], Cn = db[R + NS + n];
            const float h0 = __fmaf_rn(ex2_approx(__fmul_rn(delta0, a2[n][0])), h2.x, __fmul_rn(du0, Bn));
            const float h1 = __fmaf_rn(ex2_approx(__fmul_rn(delta1, a2[n][1])), h2.y, __fmul_rn(du1, Bn));
            y0 = __fmaf_rn(Cn, h0, y0);
            y1 = __fmaf_rn(Cn, h1, y1);
            *reinterpret_cast<float2*>(hout + (size_t)n * E) = make_float2(h0, h1);
        }
        const float o0 = __fmul_rn(__fmaf_rn(dv.x, u2.x, y0), silu_f(z2.x));
        const float o1 = __fmul_rn(__fmaf_rn(dv.y, u2.y, y1), silu_f(z2.y));
        if (f8.q) {
            // FP8 form: the row's E4M3 copy for out_proj (the CTA holds the
            // whole row), its scale from the CTA-wide maximum
            const float a = warp_max(fmaxf(fabsf(o0), fabsf(o1)));
            if ((tid & 31) == 0) red[k & 1][tid >> 5] = a;
            __syncthreads();
            float amax = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) amax = fmaxf(amax, red[k & 1][w]);
            const float inv = e4m3_row_inv(amax);
            if (tid == 0) f8.scale[s] = e4m3_row_scale(amax);
            __nv_fp8_e4m3* q = f8.q + (size_t)s * f8.Kp + c;
            q[0] = e4m3_of(o0, inv);
            q[1] = e4m3_of(o1, inv);
        } else if (yg_b) {
            *reinterpret_cast<__nv_bfloat162*>(yg_b + (size_t)s * E + c) = __floats2bfloat162_rn(o0, o1);
        } else {
            *reinterpret_cast<float2*>(yg + (size_t)s * E + c) = make_float2(o0, o1);
        }
        __syncthreads();                         // every thread is done with this stage
        if (tid == 0 && issued < mine) issue(issued++);
    }
    if (aborted && tid == 0) {
        atomicExch(err, 3);
        for (int j = k; j < issued; j++) mbar_wait(&full[j % stages], (uint32_t)((j / stages) & 1));
    }
}

}  // namespace boa
