// Microbenchmarks of the units the hot path's rooflines are quoted against:
// the MUFU ex2 rate (the scan's exp(Delta A)), the FP32 FMA rate of the
// CUDA cores (scalar and packed f32x2), the L2 read bandwidth, and the
// tcgen05.mma instruction rate per operand kind, tile width N and A source.
// Each kernel runs a long fixed stream of independent operations and is
// timed from the host with CUDA events; the MMA kernel also reports SM
// cycles per instruction from %clock64 in its issuing thread.  Inputs are
// zero or constants: only the instruction rate is measured, never a value.
#pragma once
#include "common.cuh"
#include "gemm_tc.cuh"

namespace boa {

// 2^-x chains: eight independent chains per thread keep the MUFU pipe fed;
// the values settle near 0.64 and never overflow.
__global__ void __launch_bounds__(256) k_mb_ex2(int iters, float* __restrict__ out) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = 0.01f * (float)(j + (threadIdx.x & 7));
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = ex2_approx(-x[j]);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) s = __fadd_rn(s, x[j]);
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// x <- x * 0.9999 + 1e-4 chains (eight per thread), scalar FMA.
__global__ void __launch_bounds__(256) k_mb_ffma(int iters, float* __restrict__ out) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; j++) x[j] = 0.5f + 0.01f * (float)j;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) x[j] = __fmaf_rn(x[j], 0.9999f, 1e-4f);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) s = __fadd_rn(s, x[j]);
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same chains as packed pairs: fma.rn.f32x2 does two FP32 FMAs per
// instruction (eight pairs per thread, 16 FMAs per iteration as above x 2).
__global__ void __launch_bounds__(256) k_mb_ffma2(int iters, float* __restrict__ out) {
    unsigned long long x[8];
    const unsigned long long a = ((unsigned long long)__float_as_uint(0.9999f) << 32) | __float_as_uint(0.9999f);
    const unsigned long long b = ((unsigned long long)__float_as_uint(1e-4f) << 32) | __float_as_uint(1e-4f);
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint32_t v = __float_as_uint(0.5f + 0.01f * (float)j);
        x[j] = ((unsigned long long)v << 32) | v;
    }
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[j]) : "l"(a), "l"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) s = __fadd_rn(s, __uint_as_float((uint32_t)x[j]));
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Grid-stride 16-byte reads of a buffer that stays in L2 (ld.global.cg:
// cached in L2 only, so the SMs' L1 does not serve repeats).
__global__ void __launch_bounds__(512) k_mb_l2(const float4* __restrict__ buf, size_t n4, int passes,
                                              float* __restrict__ out) {
    float acc = 0.f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; p++)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc = __fadd_rn(acc, __fadd_rn(__fadd_rn(v.x, v.y), __fadd_rn(v.z, v.w)));
        }
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// tcgen05.mma issue rate.  One CTA per SM (its shared memory request is
// more than half the SM's), 128 threads.  Operand tiles: A 128 rows x 128 B,
// B 256 rows x 128 B, both zero, K-major with the 128-byte swizzle (the
// layout the projection kernels use).  Thread 0 issues `reps` k-blocks of
// four instructions (32 bytes of K each), then commits and waits; its
// %clock64 difference over the instruction count is the SM's steady-state
// cost per instruction.
//   kind: 0 tf32, 1 f16 (BF16 operands), 2 f8f6f4 (E4M3 operands)
//   M: 128 or 64;  N: a multiple of 16 (M = 128) or 8 (M = 64), <= 256
//   flags bit 0: A from TMEM (tf32, M = 128 only)
//   flags bit 1: alternate between two accumulators (N <= 128)
//   flags bit 2: descriptors hoisted, straight-line issue (k_mb_mma_fast below)
constexpr int kMbSmemBytes = 120 * 1024;
constexpr int kMbFlagATmem = 1;
constexpr int kMbFlagTwoAcc = 2;
constexpr int kMbFlagFastIssue = 4;
constexpr int kMbFlagStages = 8;       // k_mb_mma_stages, single issuing thread
constexpr int kMbFlagStagesWarp = 16;  // k_mb_mma_stages, warp-uniform with an elected issuer

__global__ void __launch_bounds__(128, 1) k_mb_mma(int kind, int M, int N, int flags, int reps,
                                                  unsigned long long* __restrict__ cycles, int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* sa = smem;                          // 16 KB
    uint8_t* sb = smem + 16 * 1024;              // 32 KB
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 48 * 1024);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 48 * 1024 + 8);
    for (int i = threadIdx.x; i < 48 * 1024 / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int warp = threadIdx.x / 32;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t a_col = 384;                  // A operand columns when it comes from TMEM
    if (flags & kMbFlagATmem) {
        uint32_t z[16];
#pragma unroll
        for (int i = 0; i < 16; i++) z[i] = 0u;
        const uint32_t row = tmem + ((uint32_t)(32 * warp) << 16) + a_col;
        tmem_st16(row, z);
        tmem_st16(row + 16, z);
        tmem_wait_st();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x == 0) {
        const uint32_t idesc = kind == 0 ? umma_idesc_tf32(M, N) : kind == 1 ? umma_idesc_bf16(M, N)
                                                                           : umma_idesc_e4m3(M, N);
        const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
        const bool two = (flags & kMbFlagTwoAcc) != 0;
        const unsigned long long t0 = clock64();
        for (int r = 0; r < reps; r++) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int i = 4 * r + k;
                const uint32_t d = tmem + (two ? (uint32_t)((i & 1) * 128) : 0u);
                const uint32_t acc = two ? (i >= 2 ? 1u : 0u) : (i >= 1 ? 1u : 0u);
                const uint64_t bdesc = umma_desc_sw128(b0 + 32 * k);
                if (kind == 0) {
                    if (flags & kMbFlagATmem) umma_tf32_ta(d, tmem + a_col + 8 * k, bdesc, idesc, acc);
                    else umma_tf32(d, umma_desc_sw128(a0 + 32 * k), bdesc, idesc, acc);
                } else if (kind == 1) {
                    umma_bf16(d, umma_desc_sw128(a0 + 32 * k), bdesc, idesc, acc);
                } else {
                    umma_e4m3(d, umma_desc_sw128(a0 + 32 * k), bdesc, idesc, acc);
                }
            }
        }
        umma_commit(bar);
        const bool ok = mbar_wait(bar, 0);
        const unsigned long long t1 = clock64();
        cycles[blockIdx.x] = t1 - t0;
        if (!ok) {
            atomicExch(err, 1);
            mbar_wait(bar, 0);                   // once more (bounded) before TMEM is released
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// The same measurement with the issue path stripped down: the operand
// descriptors are computed once, before the timed loop, and each iteration
// issues 16 instructions in straight-line code (accumulate on after the very
// first).  Comparing it with k_mb_mma separates the tensor pipe's own cost
// per instruction from the issuing thread's descriptor arithmetic.
template <int KIND, bool ATMEM>
__global__ void __launch_bounds__(128, 1) k_mb_mma_fast(int M, int N, int reps, unsigned long long* __restrict__ cycles,
                                                       int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 48 * 1024);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 48 * 1024 + 8);
    for (int i = threadIdx.x; i < 48 * 1024 / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int warp = threadIdx.x / 32;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t a_col = 384;
    if (ATMEM) {
        uint32_t z[16];
#pragma unroll
        for (int i = 0; i < 16; i++) z[i] = 0u;
        const uint32_t row = tmem + ((uint32_t)(32 * warp) << 16) + a_col;
        tmem_st16(row, z);
        tmem_st16(row + 16, z);
        tmem_wait_st();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x == 0) {
        const uint32_t idesc = KIND == 0 ? umma_idesc_tf32(M, N) : KIND == 1 ? umma_idesc_bf16(M, N)
                                                                           : umma_idesc_e4m3(M, N);
        uint64_t ad[4], bd[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            ad[k] = umma_desc_sw128(smem_u32(smem) + 32 * k);
            bd[k] = umma_desc_sw128(smem_u32(smem + 16 * 1024) + 32 * k);
        }
        auto mma = [&](int k, uint32_t acc) {
            if (KIND == 0) {
                if (ATMEM) umma_tf32_ta(tmem, tmem + a_col + 8 * k, bd[k], idesc, acc);
                else umma_tf32(tmem, ad[k], bd[k], idesc, acc);
            } else if (KIND == 1) {
                umma_bf16(tmem, ad[k], bd[k], idesc, acc);
            } else {
                umma_e4m3(tmem, ad[k], bd[k], idesc, acc);
            }
        };
        const unsigned long long t0 = clock64();
        mma(0, 0u);
        for (int r = 0; r < reps; r++) {
#pragma unroll
            for (int j = 0; j < 16; j++) mma(j & 3, 1u);
        }
        umma_commit(bar);
        const bool ok = mbar_wait(bar, 0);
        const unsigned long long t1 = clock64();
        cycles[blockIdx.x] = t1 - t0;
        if (!ok) {
            atomicExch(err, 1);
            mbar_wait(bar, 0);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// The issue pattern of the projection kernels: k-blocks cycle through four
// shared-memory stages (A 16 KB + B 32 KB each), so the descriptors change
// every k-block.  WARP = false: one thread computes and issues; WARP = true:
// the 32 lanes of warp 0 compute the (warp-uniform) descriptors and one
// elected lane issues.
constexpr int kMbStageBytes = 48 * 1024;
constexpr int kMbStagesSmemBytes = 4 * kMbStageBytes + 2048;

template <int KIND, bool WARP>
__global__ void __launch_bounds__(128, 1) k_mb_mma_stages(int M, int N, int reps,
                                                         unsigned long long* __restrict__ cycles,
                                                         int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 4 * kMbStageBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 4 * kMbStageBytes + 8);
    for (int i = threadIdx.x; i < 4 * kMbStageBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int warp = threadIdx.x / 32;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const bool issuer_group = WARP ? warp == 0 : threadIdx.x == 0;
    if (issuer_group) {
        const uint32_t idesc = KIND == 0 ? umma_idesc_tf32(M, N) : KIND == 1 ? umma_idesc_bf16(M, N)
                                                                           : umma_idesc_e4m3(M, N);
        const bool leader = WARP ? elect_one() : true;
        const unsigned long long t0 = clock64();
        for (int kb = 0; kb < reps; kb++) {
            const uint32_t sa = smem_u32(smem + (size_t)(kb & 3) * kMbStageBytes);
            const uint32_t sb = sa + 16 * 1024;
            if (leader) {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const uint32_t acc = (kb | k) != 0 ? 1u : 0u;
                    if (KIND == 0) umma_tf32(tmem, umma_desc_sw128(sa + 32 * k), umma_desc_sw128(sb + 32 * k), idesc, acc);
                    else if (KIND == 1) umma_bf16(tmem, umma_desc_sw128(sa + 32 * k), umma_desc_sw128(sb + 32 * k), idesc, acc);
                    else umma_e4m3(tmem, umma_desc_sw128(sa + 32 * k), umma_desc_sw128(sb + 32 * k), idesc, acc);
                }
            }
            if (WARP) __syncwarp();
        }
        if (leader) umma_commit(bar);
        const bool ok = mbar_wait(bar, 0);
        const unsigned long long t1 = clock64();
        if (leader) {
            cycles[blockIdx.x] = t1 - t0;
            if (!ok) {
                atomicExch(err, 1);
                mbar_wait(bar, 0);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

}  // namespace boa
