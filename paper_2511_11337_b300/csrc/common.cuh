// Shared device-side definitions for the BOA CUDA library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace boa {

constexpr uint32_t kProbBits = 16;                 // B: CDF precision, M = 2^B
constexpr uint32_t kM = 1u << kProbBits;           // M = 65536
constexpr uint32_t kQuantScale = kM - 256;         // f_a = 1 + floor(p_a (M - 256))
constexpr uint64_t kTop = 1ull << 24;              // 2^(w-8) with w = 32
constexpr uint64_t kBot = 1ull << 16;              // straddle threshold
constexpr uint64_t kMask32 = 0xFFFFFFFFull;

// Per-stream range-coder state.  L in [0, 2^32), R in [1, 2^32] with
// L + R <= 2^32 (held in 64 bits so R = 2^32 and the products R * C fit).
struct CoderState {
    uint64_t L, R, C;     // C: decoder code value
    uint64_t pos;         // bytes written (encoder) / read (decoder), coded part only
    uint32_t flags;       // kFlag* bits
    uint32_t pad;
};

constexpr uint32_t kFlagOverflow = 1;   // encoder ran out of output capacity
constexpr uint32_t kFlagCorrupt = 2;    // decoder saw an impossible state or read past the end
constexpr uint32_t kFlagLoop = 4;       // renormalisation exceeded its proven bound

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization may start while its predecessor in the stream is still
// running: pdl_launch_next lets this kernel's successor start early (it runs
// once every CTA here has issued it), and pdl_wait_prev blocks until the
// predecessor has finished and its writes are visible.  Every kernel that
// the library launches that way calls pdl_wait_prev before it reads any
// input or writes any output.  Without that launch attribute both return
// at once.
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// 2^x on the MUFU unit (ex2.approx); used for exp(Delta * A) with A
// pre-scaled by log2(e).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// SiLU and softplus on the MUFU unit (ex2 / lg2 / rcp approximations): a
// fixed instruction sequence, so every kernel that calls them produces the
// same bits for the same input.
__device__ __forceinline__ float silu_f(float v) {
    return __fdividef(v, __fadd_rn(1.0f, __expf(-v)));
}

__device__ __forceinline__ float softplus_f(float v) {
    return v > 20.0f ? v : __logf(__fadd_rn(1.0f, __expf(v)));
}

__device__ __forceinline__ float gelu_f(float v) {
    return __fmul_rn(__fmul_rn(0.5f, v), __fadd_rn(1.0f, erff(__fmul_rn(v, 0.70710678118654752f))));
}

}  // namespace boa
