// Tensor-core GEMM for the predictor's projections on sm_103a:
//     C[M][N] = epi(A[M][K] . W[N][K]^T),  A and W in BF16, FP32 accumulation.
//
// One CTA of 128 threads owns one 128 x BN output tile:
//   - thread 0 streams K-blocks of A and W into a ring of shared-memory
//     stages with TMA (cp.async.bulk.tensor, 128-byte swizzle), signalling
//     "full" mbarriers;
//   - warp 1 walks the K blocks and one elected lane issues tcgen05.mma
//     (M = 128, N = BN, K = 16 per instruction) into a TMEM accumulator and
//     frees each stage with tcgen05.commit;
//   - all four warps then read their 32 TMEM lanes (rows) with tcgen05.ld and
//     apply the epilogue.
// Every output element sees the same instruction sequence (same K order,
// same MMA shape, same epilogue) wherever its row sits in the batch, so the
// compression and decompression passes stay bit-identical.
//
// Waits on mbarriers are bounded (about 2 s of globaltimer); on expiry the
// kernel records an error code in *err, skips the remaining work, releases
// its TMEM and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "gemm_fp32.cuh"

namespace boa {

constexpr int kTcThreads = 128;
constexpr int kTcBM = 128;
constexpr int kTcBK = 64;                  // 64 bf16 = 128 bytes = one swizzle atom row
constexpr uint64_t kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true once the phase with the given parity has completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (!mbar_try(bar, parity))
        if (globaltimer() - t0 > kWaitNs) return false;
    return true;
}

// One lane of the (converged) warp: the MMA issuers below run their loop on
// the whole warp, so the waits and descriptor arithmetic are warp-uniform
// (the uniform datapath), and only the elected lane issues instructions.
// Measured on B300: a stream of tcgen05.mma issued this way runs at the
// tensor pipe's own rate (about max(46, N / 2) SM cycles per instruction for
// M = 128 and 32 bytes of K, any operand kind), against about 72 cycles per
// instruction when one thread computes every descriptor itself.
__device__ __forceinline__ bool elect_one() {
    uint32_t pred = 0;
    asm volatile("{\n .reg .pred p;\n elect.sync _|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}\n" : "=r"(pred));
    return pred != 0;
}

// Bring a tensor map (a __grid_constant__ kernel parameter) into the TMA
// unit's descriptor cache before its first use.
__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major tile written by TMA with the
// 128-byte swizzle; rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);         // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for SW128 K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                          // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                          // swizzle mode: 128B
    return d;
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4)                      // D format F32
         | (1u << 7)                      // A format BF16
         | (1u << 10)                     // B format BF16
         | ((uint32_t)(N >> 3) << 17)     // N / 8
         | ((uint32_t)(M >> 4) << 24);    // M / 16
}

// Instruction descriptor, kind::f8f6f4: E4M3 x E4M3 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t umma_idesc_e4m3(int M, int N) {
    return (1u << 4)                      // D format F32
         | (0u << 7)                      // A format E4M3
         | (0u << 10)                     // B format E4M3
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_e4m3(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Operand kinds of the 128-byte-per-row tensor-core kernel.
enum TcKind : int { kKindBF16 = 0, kKindE4M3 = 1 };

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16 consecutive 32-bit TMEM columns of the warp's 32 lanes (one lane per
// thread), the store counterpart of tmem_ld16_nowait.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Epilogue shared by the tensor-core kernels.  Warp q owns accumulator rows
// (TMEM lanes) 32q .. 32q+31.  Phase 1 (tc_stage_tile): it copies them, 16
// columns per tcgen05.ld, into its own slice of the (now idle) pipeline
// shared memory, 16-byte chunks XOR-swizzled by row so the writes are
// conflict-free.  Phase 2 (tc_store_rows): a warp walks a range of rows,
// each lane taking one 16-byte chunk, so every global store of the warp
// covers whole contiguous row segments; the epilogue arithmetic (scales,
// bias, GELU, residual) happens here.  With split K (a cluster of `peers`
// CTAs along z, each with the partial sum of its share of the K blocks) the
// chunk is the sum of the peers' staged tiles, read through distributed
// shared memory in rank order 0, 1, ..., so every element sees the same
// additions wherever its tile runs.
// row_scale / col_scale (FP8 operands): acc * row_scale[m] * col_scale[n].
template <int BN>
struct TileLayout {
    static constexpr int kChunks = BN / 16;
    static constexpr int kSlots = BN / 4;                       // float4 per row
    static constexpr int kMask = kSlots >= 16 ? 7 : 3;          // swizzle stays inside the row
    static constexpr int kLaneSlots = kSlots < 32 ? kSlots : 32;   // float4 columns one pass covers
    static constexpr int kPasses = kSlots / kLaneSlots;         // column passes per row (2 for BN = 256)
    static constexpr int kRowsPerIter = 32 / kLaneSlots;        // rows one warp store covers
};

// ROLLED: one group of four loads in flight at a time (a persistent kernel
// calls this inside its tile loop, where the unrolled groups would hold
// 128 registers at once).
template <int BN, bool ROLLED = false>
__device__ __forceinline__ void tc_stage_tile(uint32_t tmem, int q, int lane, float* stage) {
    using T = TileLayout<BN>;
    float4* st = reinterpret_cast<float4*>(stage) + (size_t)q * 32 * T::kSlots;
#pragma unroll (ROLLED ? 1 : (T::kChunks + 3) / 4)
    for (int g0 = 0; g0 < T::kChunks; g0 += 4) {
        uint32_t r[4][16];
#pragma unroll
        for (int c = 0; c < 4; c++)
            if (g0 + c < T::kChunks)
                tmem_ld16_nowait(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(16 * (g0 + c)), r[c]);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if (g0 + c >= T::kChunks) break;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int f = (g0 + c) * 4 + j;
                st[lane * T::kSlots + (f ^ (lane & T::kMask))] =
                    make_float4(__uint_as_float(r[c][4 * j]), __uint_as_float(r[c][4 * j + 1]),
                                __uint_as_float(r[c][4 * j + 2]), __uint_as_float(r[c][4 * j + 3]));
            }
        }
    }
}

// Split K inside one CTA: the K blocks fall into `chunks` consecutive
// chunks, each accumulated in its own TMEM columns (chunk j at column
// j * chunk_cols), and the staged tile is their sum in chunk order 0, 1, ...
// This is the same sum, with the same additions, as a cluster of `chunks`
// CTAs each holding one chunk (tc_store_rows with peers = chunks).
template <int BN>
__device__ __forceinline__ void tc_stage_tile_sum(uint32_t tmem, int q, int lane, float* stage, int chunks,
                                                  int chunk_cols) {
    using T = TileLayout<BN>;
    float4* st = reinterpret_cast<float4*>(stage) + (size_t)q * 32 * T::kSlots;
    const uint32_t base = tmem + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
    for (int g0 = 0; g0 < T::kChunks; g0 += 2) {
        float acc[2][16];
        uint32_t r[2][16];
#pragma unroll 1
        for (int j = 0; j < chunks; j++) {
#pragma unroll
            for (int c = 0; c < 2; c++)
                if (g0 + c < T::kChunks) tmem_ld16_nowait(base + (uint32_t)(j * chunk_cols + 16 * (g0 + c)), r[c]);
            tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 2; c++)
#pragma unroll
                for (int i = 0; i < 16; i++)
                    acc[c][i] = j == 0 ? __uint_as_float(r[c][i]) : __fadd_rn(acc[c][i], __uint_as_float(r[c][i]));
        }
#pragma unroll
        for (int c = 0; c < 2; c++) {
            if (g0 + c >= T::kChunks) break;
#pragma unroll
            for (int jj = 0; jj < 4; jj++) {
                const int f = (g0 + c) * 4 + jj;
                st[lane * T::kSlots + (f ^ (lane & T::kMask))] =
                    make_float4(acc[c][4 * jj], acc[c][4 * jj + 1], acc[c][4 * jj + 2], acc[c][4 * jj + 3]);
            }
        }
    }
}

constexpr int kMaxPeers = 4;                      // split-K factors are 1, 2 or 4

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t dsmem_addr(const void* local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
    return r;
}

__device__ __forceinline__ float4 dsmem_ld4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ int dsmem_ld_s32(uint32_t addr) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// Rows r_beg .. r_beg + n_rows - 1 of the staged tile (n_rows a multiple of
// the rows one warp store covers) to global memory.
template <int BN, int EPI>
__device__ __forceinline__ void tc_store_rows(int r_beg, int n_rows, int lane, int m0, int n0, int M, int N,
                                              const float* __restrict__ bias, float* __restrict__ Cm,
                                              __nv_bfloat16* __restrict__ out_bf16, const float* stage, int peers,
                                              const float* __restrict__ row_scale,
                                              const float* __restrict__ col_scale) {
    using T = TileLayout<BN>;
    const float4* st = reinterpret_cast<const float4*>(stage);
    const int kIters = n_rows / T::kRowsPerIter;
#pragma unroll 1
    for (int pass = 0; pass < T::kPasses; pass++) {
    const int f = lane % T::kLaneSlots + pass * T::kLaneSlots;
    const bool active = lane < T::kRowsPerIter * T::kLaneSlots;
    const int n = n0 + 4 * f;
    const bool col_ok = active && n < N;                 // N % 4 == 0
    float4 bv = make_float4(0.f, 0.f, 0.f, 0.f), cs = make_float4(1.f, 1.f, 1.f, 1.f);
    if (col_ok && (EPI == kEpiBias || EPI == kEpiBiasGelu || EPI == kEpiBiasResid))
        bv = *reinterpret_cast<const float4*>(bias + n);
    if (col_ok && col_scale) cs = *reinterpret_cast<const float4*>(col_scale + n);
    constexpr bool kResid = EPI == kEpiResid || EPI == kEpiBiasResid;
    // rows whose residual loads are in flight together
    constexpr int kBatch = kResid && T::kRowsPerIter == 2 ? 16 : 8;
#pragma unroll 1
    for (int it0 = 0; it0 < kIters; it0 += kBatch) {
        float4 old[kBatch];
        float rsv[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; u++) {
            const int rl = r_beg + (it0 + u) * T::kRowsPerIter + lane / T::kLaneSlots;
            const int row = m0 + rl;
            old[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            rsv[u] = 1.f;
            if (it0 + u < kIters && col_ok && row < M) {
                if (kResid) old[u] = *reinterpret_cast<const float4*>(Cm + (size_t)row * N + n);
                if (row_scale) rsv[u] = row_scale[row];
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; u++) {
            if (it0 + u >= kIters) break;
            const int rl = r_beg + (it0 + u) * T::kRowsPerIter + lane / T::kLaneSlots;
            const int row = m0 + rl;
            if (!col_ok || row >= M) continue;
            const float4* src = st + rl * T::kSlots + (f ^ (rl & T::kMask));
            float4 a;
            if (peers == 1) {
                a = *src;
            } else {
                // all peers' chunks requested at once, then added in rank order
                float4 pv[kMaxPeers];
#pragma unroll
                for (int p = 0; p < kMaxPeers; p++)
                    if (p < peers) pv[p] = dsmem_ld4(dsmem_addr(src, (uint32_t)p));
                a = pv[0];
#pragma unroll
                for (int p = 1; p < kMaxPeers; p++)
                    if (p < peers) {
                        a.x = __fadd_rn(a.x, pv[p].x);
                        a.y = __fadd_rn(a.y, pv[p].y);
                        a.z = __fadd_rn(a.z, pv[p].z);
                        a.w = __fadd_rn(a.w, pv[p].w);
                    }
            }
            float o[4] = {a.x, a.y, a.z, a.w};
            const float* bp = reinterpret_cast<const float*>(&bv);
            const float* cp = reinterpret_cast<const float*>(&cs);
            const float* op = reinterpret_cast<const float*>(&old[u]);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                float x = o[j];
                if (row_scale) x = __fmul_rn(__fmul_rn(x, rsv[u]), cp[j]);
                if (EPI == kEpiBias || EPI == kEpiBiasGelu || EPI == kEpiBiasResid) x = __fadd_rn(x, bp[j]);
                if (EPI == kEpiBiasGelu) x = gelu_f(x);
                if (kResid) x = __fadd_rn(op[j], x);
                o[j] = x;
            }
            *reinterpret_cast<float4*>(Cm + (size_t)row * N + n) = make_float4(o[0], o[1], o[2], o[3]);
            if (out_bf16) {
                __nv_bfloat162* bo = reinterpret_cast<__nv_bfloat162*>(out_bf16 + (size_t)row * N + n);
                bo[0] = __floats2bfloat162_rn(o[0], o[1]);
                bo[1] = __floats2bfloat162_rn(o[2], o[3]);
            }
        }
    }
    }
}

// The whole epilogue of one CTA.  Every thread of the CTA calls it (the
// cluster barriers of split K count every thread); `epi` marks the four
// epilogue warps and q their TMEM quadrant.  bad: this CTA's pipeline gave
// up; with split K no CTA of the cluster then stores anything.  chunks > 1
// (only without a cluster): split K held in this CTA's TMEM, see
// tc_stage_tile_sum.
template <int BN, int EPI>
__device__ __forceinline__ void tc_epilogue(bool epi, bool bad, int* bad_flag, uint32_t tmem, int q, int lane, int m0,
                                            int n0, int M, int N, const float* __restrict__ bias,
                                            float* __restrict__ Cm, __nv_bfloat16* __restrict__ out_bf16,
                                            float* stage, const float* __restrict__ row_scale = nullptr,
                                            const float* __restrict__ col_scale = nullptr, int chunks = 1,
                                            int chunk_cols = 0, int peers = -1) {
    if (peers < 0) peers = (int)gridDim.z;
    if (peers == 1) {
        if (epi && !bad) {
            if (chunks > 1) tc_stage_tile_sum<BN>(tmem, q, lane, stage, chunks, chunk_cols);
            else tc_stage_tile<BN>(tmem, q, lane, stage);
            __syncwarp();
            tc_store_rows<BN, EPI>(32 * q, 32, lane, m0, n0, M, N, bias, Cm, out_bf16, stage, 1, row_scale,
                                   col_scale);
        }
        return;
    }
    if (epi && !bad) tc_stage_tile<BN>(tmem, q, lane, stage);
    if (threadIdx.x == 0) *bad_flag = bad ? 1 : 0;
    __syncwarp();
    cluster_sync_all();                                  // every peer's tile and flag are in place
    bool any_bad = false;
    for (int p = 0; p < peers; p++) any_bad |= dsmem_ld_s32(dsmem_addr(bad_flag, (uint32_t)p)) != 0;
    if (epi && !any_bad) {
        const int rows = kTcBM / peers;                  // this CTA's share of the tile
        const int per_warp = rows / 4;
        tc_store_rows<BN, EPI>((int)cluster_rank() * rows + q * per_warp, per_warp, lane, m0, n0, M, N, bias, Cm,
                               out_bf16, stage, peers, row_scale, col_scale);
    }
    cluster_sync_all();                                  // peers are done reading this CTA's tile
}

// DEEP = false: about 110 KB of stages so that two CTAs share an SM (one's
// epilogue overlaps the other's loads and MMAs; TMEM 2 x kTmemCols <= 512).
// DEEP = true: up to about 200 KB (one CTA per SM), for grids smaller than
// the SM count, where every K block's loads should be in flight at once.
// The stage count never changes the MMA sequence, only the overlap.
template <int BN, bool DEEP = false>
struct TcSmem {
    static constexpr int kA = kTcBM * kTcBK * 2;     // 16 KB
    static constexpr int kB = BN * kTcBK * 2;
    static constexpr int kStage = kA + kB;
    static constexpr int kStagesRaw = ((DEEP ? 200 : 110) * 1024) / kStage;
    // the epilogue stages the 128 x BN FP32 tile in the same memory
    static constexpr int kStagesTile = (kTcBM * BN * 4 + kStage - 1) / kStage;
    static constexpr int kStagesMin = kStagesTile > 2 ? kStagesTile : 2;
    static constexpr int kStages = kStagesRaw < kStagesMin ? kStagesMin : (kStagesRaw > 8 ? 8 : kStagesRaw);
    static constexpr int kTmemCols = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    // stages, then barriers (full, empty, done) and the TMEM address slot
    static constexpr int kBars = 2 * kStages + 1;
    static constexpr size_t kBytes = 1024 /*alignment slack*/ + (size_t)kStages * kStage + 8 * kBars + 16;
};

// out_bf16 (optional): a BF16 copy of the stored result (feeds the next GEMM).
// KIND selects BF16 operands (K = 64 per stage, kind::f16) or E4M3 operands
// (K = 128 per stage, kind::f8f6f4, with row / column scales in the
// epilogue); either way a stage row is 128 bytes.
template <int BN, int EPI, int KIND, bool DEEP = false>
__global__ void __launch_bounds__(kTcThreads)
k_gemm_tc_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const float* __restrict__ bias, float* __restrict__ Cm, __nv_bfloat16* __restrict__ out_bf16,
               int M, int N, int K, int* __restrict__ err, const float* __restrict__ row_scale,
               const float* __restrict__ col_scale, int chunks, int zpart) {
    constexpr int kElemK = KIND == kKindE4M3 ? 128 : kTcBK;    // elements per 128-byte stage row
    using L = TcSmem<BN, DEEP>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)L::kStages * L::kStage);
    uint64_t* full = bars;
    uint64_t* empty = bars + L::kStages;
    uint64_t* done = bars + 2 * L::kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + L::kBars);
    __shared__ int abort_flag;

    __shared__ int bad_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * BN;
    const int nk = K / kElemK / (int)gridDim.z;          // split K: this CTA's K blocks
    const int kb0 = (int)blockIdx.z * nk;
    const int nkc = nk / chunks;                         // K blocks per TMEM chunk
    const uint32_t tmem_cols = (uint32_t)(L::kTmemCols * chunks);

    if (threadIdx.x == 0) {
        tma_prefetch_map(&tmA);
        tma_prefetch_map(&tmB);
        abort_flag = 0;
        for (int i = 0; i < L::kBars; i++) mbar_init(&bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // The set-up above overlaps the previous kernel.  B (the weights) is
    // never written by the kernel that precedes a projection, so the first
    // stages' B tiles are requested before waiting for it; A only after.
    pdl_launch_next();
    const int pre = nk < L::kStages ? nk : L::kStages;
    if (threadIdx.x == 0)
        for (int kb = 0; kb < pre; kb++) {
            mbar_expect_tx(&full[kb], L::kStage);
            tma_load_2d(&tmB, &full[kb], smem + (size_t)kb * L::kStage + L::kA, (kb0 + kb) * kElemK, n0);
        }
    pdl_wait_prev();

    int armed_last = -1;   // producer: last K-block whose loads were issued
    if (threadIdx.x == 0) {
        // TMA producer
        for (int kb = 0; kb < nk; kb++) {
            const int s = kb % L::kStages;
            uint8_t* sa = smem + (size_t)s * L::kStage;
            if (kb >= pre) {
                if (!mbar_wait(&empty[s], ((kb / L::kStages) - 1) & 1)) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
                mbar_expect_tx(&full[s], L::kStage);
                tma_load_2d(&tmB, &full[s], sa + L::kA, (kb0 + kb) * kElemK, n0);
            }
            tma_load_2d(&tmA, &full[s], sa, (kb0 + kb) * kElemK, m0);
            armed_last = kb;
        }
    } else if (warp == 1) {
        // MMA issuer: the whole warp walks the K blocks, one lane issues
        constexpr uint32_t idesc = KIND == kKindE4M3 ? umma_idesc_e4m3(kTcBM, BN) : umma_idesc_bf16(kTcBM, BN);
        const bool leader = elect_one();
        // descriptors of stage 0's first 32 bytes of K; stage s and K step k
        // add (s * kStage + 32 k) / 16 to the start-address field
        const uint64_t da0 = umma_desc_sw128(smem_u32(smem));
        const uint64_t db0 = umma_desc_sw128(smem_u32(smem + L::kA));
        bool ok = true;
        int kc = 0, chunk = 0;                           // K block within its TMEM chunk, chunk index
        for (int kb = 0; kb < nk; kb++) {
            const int s = kb % L::kStages;
            ok = __all_sync(0xffffffffu, mbar_wait(&full[s], (kb / L::kStages) & 1));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t so = (uint64_t)((s * L::kStage) >> 4);
            const uint32_t d = tmem + (uint32_t)(chunk * L::kTmemCols);
            if (leader) {
#pragma unroll
                for (int k = 0; k < 4; k++) {   // 32 bytes of K per instruction: 16 BF16 or 32 E4M3
                    if (KIND == kKindE4M3)
                        umma_e4m3(d, da0 + so + 2 * k, db0 + so + 2 * k, idesc, (kc | k) != 0 ? 1u : 0u);
                    else
                        umma_bf16(d, da0 + so + 2 * k, db0 + so + 2 * k, idesc, (kc | k) != 0 ? 1u : 0u);
                }
                umma_commit(&empty[s]);
            }
            __syncwarp();
            if (++kc == nkc) {
                kc = 0;
                chunk++;
            }
        }
        if (leader) {
            if (!ok) atomicExch(&abort_flag, 1);
            umma_commit(&done[0]);
        }
    }

    // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w + 31
    const bool finished = mbar_wait(&done[0], 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    const bool bad = !finished || abort_flag;
    if (bad && threadIdx.x == 0) {
        atomicExch(err, 1);
        // let copies and MMAs still in flight land before TMEM and shared
        // memory are released (each wait again bounded)
        for (int kb = armed_last; kb >= 0 && kb > armed_last - L::kStages; kb--)
            mbar_wait(&full[kb % L::kStages], (kb / L::kStages) & 1);
        if (!finished) mbar_wait(&done[0], 0);
    }
    // zpart: the z slices of the grid are independent parts of the K range,
    // each written to its own [M][N] output (Cm + z M N), not split K
    if (zpart) Cm += (size_t)blockIdx.z * M * N;
    tc_epilogue<BN, EPI>(true, bad, &bad_flag, tmem, warp, lane, m0, n0, M, N, bias, Cm, out_bf16,
                         reinterpret_cast<float*>(smem), row_scale, col_scale, chunks, L::kTmemCols,
                         zpart ? 1 : (int)gridDim.z);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// ------------------------------------------------------------ 3xTF32 form
//
// FP32-accurate projections on the tensor cores: every operand x is split
// into x_hi = tf32(x) (round to nearest) and x_lo = x - x_hi, and
//     A . W^T ~= A_hi W_hi^T + A_hi W_lo^T + A_lo W_hi^T
// is accumulated in FP32 in TMEM (kind::tf32, K = 8 per instruction), the
// three products of each K step always in that order.  The weights arrive
// pre-split (B_hi, B_lo in shared memory by TMA); A arrives as FP32 by TMA,
// and four converter warps split each stage's rows into A_hi and A_lo in
// TMEM (each thread its row, in its lane), where the MMAs read their A
// operand.  TMEM holds the accumulator(s) in its first columns and the A
// stages after them.  Warps: 0 TMA, 1 MMA (one elected lane issues), 2-5
// converters (with DEEP also 6-9: then 2-5 take the even K blocks and 6-9
// the odd ones), then 2-5 run the epilogue.

// Warps: 0 TMA, 1 MMA, then 4 converter warps per converter set.  A CTA
// alone on its SM (DEEP, decode-size grids) runs two sets so that two stages
// are converted at once; two CTAs sharing an SM run one set each.
__host__ __device__ constexpr int t3_threads(bool deep) { return deep ? 320 : 192; }
constexpr int kT3BK = 32;                  // 32 fp32 = 128 bytes = one swizzle atom row

__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
    return (1u << 4)                      // D format F32
         | (2u << 7)                      // A format TF32
         | (2u << 10)                     // B format TF32
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// The same MMA with A read from TMEM (row i of A in lane i, one 32-bit
// column per K element) instead of shared memory.
__device__ __forceinline__ void umma_tf32_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
        ::"r"(tmem_d), "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int BN, bool DEEP = false>
struct T3Smem {
    static constexpr int kA = kTcBM * kT3BK * 4;     // 16 KB: the FP32 A tile as TMA writes it
    static constexpr int kB = BN * kT3BK * 4;
    static constexpr int kStage = kA + 2 * kB;       // A, B_hi, B_lo (A_hi and A_lo go to TMEM)
    // two CTAs per SM with two stages each where they fit (BN <= 64);
    // otherwise (deep grids, or BN >= 128) one CTA with up to ~200 KB of stages
    static constexpr bool kOnePerSm = DEEP || 2 * kStage > 110 * 1024;
    static constexpr int kTmemCols = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;   // per K chunk
    static constexpr int kACols = 2 * kT3BK;         // TMEM columns of one stage's A_hi | A_lo
    static constexpr int kStagesSmem = kOnePerSm ? ((200 * 1024) / kStage > 8 ? 8 : (200 * 1024) / kStage) : 2;
    static constexpr int kStagesTmem = (512 - kTmemCols) / kACols;
    static constexpr int kStages = kStagesSmem < kStagesTmem ? kStagesSmem : kStagesTmem;
    static constexpr int kBars = 3 * kStages + 1;    // full, converted, empty, done
    static constexpr size_t kBytesUsed = 1024 + (size_t)kStages * kStage + 8 * kBars + 16;
    // Shared memory also caps how many CTAs share an SM's 512 TMEM columns:
    // a two-per-SM CTA asks for at least 100 KB, so at most two are resident
    // (each allocating <= 256 columns), and a one-per-SM CTA more than half
    // the SM.  Without that cap the CTAs of a split-K cluster could wait on
    // each other while a peer waits in tcgen05.alloc.
    static constexpr size_t kBytes = kOnePerSm || kBytesUsed >= 100 * 1024 ? kBytesUsed : 100 * 1024;
    static_assert((size_t)kStages * kStage >= (size_t)kTcBM * BN * 4, "the epilogue stages the tile here");
    __host__ __device__ static constexpr uint32_t pow2_cols(uint32_t n) {
        return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512;
    }
};

template <int BN, int EPI, bool DEEP = false>
__global__ void __launch_bounds__(t3_threads(DEEP))
k_gemm_tc_tf32x3(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBhi,
                 const __grid_constant__ CUtensorMap tmBlo, const float* __restrict__ bias, float* __restrict__ Cm,
                 int M, int N, int K, int* __restrict__ err, int chunks) {
    using L = T3Smem<BN, DEEP>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)L::kStages * L::kStage);
    uint64_t* full = bars;
    uint64_t* conv = bars + L::kStages;
    uint64_t* empty = bars + 2 * L::kStages;
    uint64_t* done = bars + 3 * L::kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + L::kBars);
    __shared__ int abort_flag;

    __shared__ int bad_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * BN;
    const int nk = K / kT3BK / (int)gridDim.z;           // split K: this CTA's K blocks
    const int kb0 = (int)blockIdx.z * nk;
    const int nkc = nk / chunks;                         // K blocks per TMEM chunk
    const uint32_t a_col0 = (uint32_t)(L::kTmemCols * chunks);   // first A stage's TMEM column
    const uint32_t tmem_cols = L::pow2_cols(a_col0 + (uint32_t)(L::kStages * L::kACols));

    if (threadIdx.x == 0) {
        tma_prefetch_map(&tmA);
        tma_prefetch_map(&tmBhi);
        tma_prefetch_map(&tmBlo);
        abort_flag = 0;
        for (int i = 0; i < L::kStages; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&conv[i], 128);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&done[0], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // The set-up above overlaps the previous kernel.  B_hi / B_lo (the
    // weights) are never written by the kernel that precedes a projection,
    // so the first stages' B tiles are requested before waiting for it; A
    // only after.
    pdl_launch_next();
    const int pre = nk < L::kStages ? nk : L::kStages;
    if (threadIdx.x == 0)
        for (int kb = 0; kb < pre; kb++) {
            uint8_t* st = smem + (size_t)kb * L::kStage;
            mbar_expect_tx(&full[kb], L::kStage);
            tma_load_2d(&tmBhi, &full[kb], st + L::kA, (kb0 + kb) * kT3BK, n0);
            tma_load_2d(&tmBlo, &full[kb], st + L::kA + L::kB, (kb0 + kb) * kT3BK, n0);
        }
    pdl_wait_prev();

    int armed_last = -1;
    if (threadIdx.x == 0) {
        for (int kb = 0; kb < nk; kb++) {
            const int s = kb % L::kStages;
            uint8_t* st = smem + (size_t)s * L::kStage;
            if (kb >= pre) {
                if (!mbar_wait(&empty[s], ((kb / L::kStages) - 1) & 1)) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
                mbar_expect_tx(&full[s], L::kStage);
                tma_load_2d(&tmBhi, &full[s], st + L::kA, (kb0 + kb) * kT3BK, n0);
                tma_load_2d(&tmBlo, &full[s], st + L::kA + L::kB, (kb0 + kb) * kT3BK, n0);
            }
            tma_load_2d(&tmA, &full[s], st, (kb0 + kb) * kT3BK, m0);
            armed_last = kb;
        }
    } else if (warp == 1) {
        // MMA issuer: the whole warp walks the K blocks, one lane issues
        constexpr uint32_t idesc = umma_idesc_tf32(kTcBM, BN);
        const bool leader = elect_one();
        // B_hi descriptor of stage 0's first 32 bytes of K; stage s, B_lo and
        // K step k add (s * kStage [+ kB] + 32 k) / 16 to the start address
        const uint64_t dh0 = umma_desc_sw128(smem_u32(smem + L::kA));
        bool ok = true;
        int kc = 0, chunk = 0;                           // K block within its TMEM chunk, chunk index
        for (int kb = 0; kb < nk; kb++) {
            const int s = kb % L::kStages;
            ok = __all_sync(0xffffffffu, mbar_wait(&conv[s], (kb / L::kStages) & 1));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t dh = dh0 + (uint64_t)((s * L::kStage) >> 4);
            const uint64_t dl = dh + (uint64_t)(L::kB >> 4);
            const uint32_t ahi = tmem + a_col0 + (uint32_t)(s * L::kACols);   // TMEM: A_hi | A_lo
            const uint32_t alo = ahi + kT3BK;
            const uint32_t d = tmem + (uint32_t)(chunk * L::kTmemCols);
            if (leader) {
#pragma unroll
                for (int k = 0; k < kT3BK / 8; k++) {
                    // 8 TF32 of K: 32 bytes of B (2 descriptor units), 8 TMEM columns of A
                    umma_tf32_ta(d, ahi + 8 * k, dh + 2 * k, idesc, (kc | k) != 0 ? 1u : 0u);
                    umma_tf32_ta(d, ahi + 8 * k, dl + 2 * k, idesc, 1u);
                    umma_tf32_ta(d, alo + 8 * k, dh + 2 * k, idesc, 1u);
                }
                umma_commit(&empty[s]);
            }
            __syncwarp();
            if (++kc == nkc) {
                kc = 0;
                chunk++;
            }
        }
        if (leader) {
            if (!ok) atomicExch(&abort_flag, 1);
            umma_commit(&done[0]);
        }
    } else if (warp >= 2) {
        // converters: thread (quadrant q = warp % 4, lane) takes A row
        // 32 q + lane of each of its stages (with two sets, warps 2-5 the
        // even K blocks and 6-9 the odd ones), splits it into hi and lo, and
        // writes both into its TMEM lane: A_hi in the stage's columns 0..31,
        // A_lo in 32..63
        constexpr int kSets = (t3_threads(DEEP) - 64) / 128;
        const int q = warp % 4;
        const int r = 32 * q + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + a_col0;
        for (int kb = (warp - 2) / 4; kb < nk; kb += kSets) {
            const int s = kb % L::kStages;
            if (!mbar_wait(&full[s], (kb / L::kStages) & 1)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            // the stage's TMEM columns were last read by MMAs that completed
            // before this stage's loads were issued
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // row r of the 128-byte-swizzled tile: 16-byte chunk c sits at
            // chunk position c ^ (r % 8)
            const uint8_t* row = smem + (size_t)s * L::kStage + (size_t)r * 128;
#pragma unroll
            for (int half = 0; half < 2; half++) {
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const int ch = 4 * half + c;
                    const float4 v = *reinterpret_cast<const float4*>(row + ((ch ^ (r & 7)) << 4));
                    const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const float h = tf32_rna(x[e]);
                        hi[4 * c + e] = __float_as_uint(h);
                        lo[4 * c + e] = __float_as_uint(__fsub_rn(x[e], h));
                    }
                }
                const uint32_t col = trow + (uint32_t)(s * L::kACols + 16 * half);
                tmem_st16(col, hi);
                tmem_st16(col + kT3BK, lo);
            }
            tmem_wait_st();
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&conv[s])) : "memory");
        }
    }

    const bool finished = mbar_wait(&done[0], 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    const bool bad = !finished || abort_flag;
    if (bad && threadIdx.x == 0) {
        atomicExch(err, 1);
        for (int kb = armed_last; kb >= 0 && kb > armed_last - L::kStages; kb--)
            mbar_wait(&full[kb % L::kStages], (kb / L::kStages) & 1);
        if (!finished) mbar_wait(&done[0], 0);
    }
    tc_epilogue<BN, EPI>(warp >= 2 && warp < 6, bad, &bad_flag, tmem, warp % 4, lane, m0, n0, M, N, bias, Cm,
                         nullptr, reinterpret_cast<float*>(smem), nullptr, nullptr, chunks, L::kTmemCols);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// ------------------------------------------------ persistent 3xTF32 GEMM
//
// Compression-size projections without split K (in_proj, out_proj, head):
// one CTA per SM walks the 128 x 128 output tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... (row-block major, so consecutive tiles share
// their A rows).  The TMA producer, the converters and the MMA issuer stream
// K blocks across tile boundaries through one ring of stages; the MMAs
// accumulate tile j in TMEM accumulator j % 2, and four epilogue warps of
// their own drain the other accumulator through a dedicated staging buffer
// meanwhile.  Each tile sees the MMA sequence and epilogue arithmetic of
// k_gemm_tc_tf32x3 (same K order, same 3xTF32 products, same stores), so
// the bits are the same as the per-tile kernel's.
//
// Warps: 0 TMA, 1 MMA (one elected lane issues), 2-5 converters, 6-9
// epilogue.  Barriers: full / conv / empty per stage as in the per-tile
// kernel; acc_full[b] (the MMAs of accumulator b's tile have completed) and
// acc_empty[b] (the epilogue has read accumulator b).  Waits are bounded:
// on expiry the CTA records the error, lets the copies and MMAs it issued
// land (bounded again), releases TMEM and returns.
struct T3P {
    static constexpr int BN = 128;
    static constexpr int kA = kTcBM * kT3BK * 4;                 // 16 KB of FP32 A per stage
    static constexpr int kB = BN * kT3BK * 4;                    // 16 KB each of B_hi, B_lo
    static constexpr int kStage = kA + 2 * kB;
    static constexpr int kStages = 3;
    static constexpr int kStaging = kTcBM * BN * 4;              // 64 KB: the epilogue's tile
    static constexpr int kACols = 2 * kT3BK;
    static constexpr uint32_t kAccCols = BN;                     // two accumulators: columns 0, 128
    static constexpr uint32_t kACol0 = 2 * kAccCols;             // A stages after them
    static constexpr uint32_t kTmemCols = 512;
    static constexpr int kBars = 3 * kStages + 4 + 1;            // full, conv, empty; acc_full[2], acc_empty[2]; mma_done
    static constexpr size_t kBytes = 1024 + (size_t)kStages * kStage + kStaging + 8 * kBars + 16;
    static constexpr int kThreads = 320;
    static_assert(kACol0 + kStages * kACols <= kTmemCols, "accumulators and A stages fit the SM's TMEM");
};

template <int EPI>
__global__ void __launch_bounds__(T3P::kThreads, 1)
k_gemm_t3_persist(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBhi,
                  const __grid_constant__ CUtensorMap tmBlo, const float* __restrict__ bias, float* __restrict__ Cm,
                  int M, int N, int K, int* __restrict__ err) {
    using L = T3P;
    constexpr int S = L::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    float* staging = reinterpret_cast<float*>(smem + (size_t)S * L::kStage);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * L::kStage + L::kStaging);
    uint64_t* full = bars;
    uint64_t* conv = bars + S;
    uint64_t* empty = bars + 2 * S;
    uint64_t* acc_full = bars + 3 * S;
    uint64_t* acc_empty = bars + 3 * S + 2;
    uint64_t* mma_done = bars + 3 * S + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + L::kBars);
    __shared__ int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int tiles_n = (N + L::BN - 1) / L::BN;
    const int n_tiles = tiles_n * ((M + kTcBM - 1) / kTcBM);
    const int nk = K / kT3BK;

    if (threadIdx.x == 0) {
        tma_prefetch_map(&tmA);
        tma_prefetch_map(&tmBhi);
        tma_prefetch_map(&tmBlo);
        abort_flag = 0;
        for (int i = 0; i < S; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&conv[i], 128);
            mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
        }
        mbar_init(mma_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(L::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    pdl_launch_next();
    pdl_wait_prev();

    int issued = 0;                                // producer: K blocks whose loads went out
    if (threadIdx.x == 0) {
        // TMA producer
        int g = 0;
#pragma unroll 1
        for (int t = blockIdx.x; t < n_tiles && !*(volatile int*)&abort_flag; t += gridDim.x) {
            const int m0 = (t / tiles_n) * kTcBM, n0 = (t % tiles_n) * L::BN;
#pragma unroll 1
            for (int kb = 0; kb < nk; kb++, g++) {
                const int s = g % S;
                if (g >= S && !mbar_wait(&empty[s], (uint32_t)(((g / S) - 1) & 1))) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
                uint8_t* st = smem + (size_t)s * L::kStage;
                mbar_expect_tx(&full[s], L::kStage);
                tma_load_2d(&tmA, &full[s], st, kb * kT3BK, m0);
                tma_load_2d(&tmBhi, &full[s], st + L::kA, kb * kT3BK, n0);
                tma_load_2d(&tmBlo, &full[s], st + L::kA + L::kB, kb * kT3BK, n0);
                issued = g + 1;
            }
        }
    } else if (warp >= 2 && warp < 6) {
        // converters: thread (quadrant q, lane) splits row 32 q + lane of
        // every stage into A_hi / A_lo in its TMEM lane
        const int q = warp % 4;
        const int r = 32 * q + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + L::kACol0;
        int g = 0;
        bool ok = true;
#pragma unroll 1
        for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
#pragma unroll 1
            for (int kb = 0; kb < nk; kb++, g++) {
                const int s = g % S;
                if (!mbar_wait(&full[s], (uint32_t)((g / S) & 1))) {
                    atomicExch(&abort_flag, 1);
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint8_t* row = smem + (size_t)s * L::kStage + (size_t)r * 128;
#pragma unroll
                for (int half = 0; half < 2; half++) {
                    uint32_t hi[16], lo[16];
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const int ch = 4 * half + c;
                        const float4 v = *reinterpret_cast<const float4*>(row + ((ch ^ (r & 7)) << 4));
                        const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            const float h = tf32_rna(x[e]);
                            hi[4 * c + e] = __float_as_uint(h);
                            lo[4 * c + e] = __float_as_uint(__fsub_rn(x[e], h));
                        }
                    }
                    const uint32_t col = trow + (uint32_t)(s * L::kACols + 16 * half);
                    tmem_st16(col, hi);
                    tmem_st16(col + kT3BK, lo);
                }
                tmem_wait_st();
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&conv[s])) : "memory");
            }
        }
    }
    else if (warp == 1) {
        // MMA issuer: tile j accumulates in accumulator j % 2, after the
        // epilogue has read that accumulator's previous tile (j - 2)
        constexpr uint32_t idesc = umma_idesc_tf32(kTcBM, L::BN);
        const bool leader = elect_one();
        const uint64_t dh0 = umma_desc_sw128(smem_u32(smem + L::kA));
        bool ok = true;
        int g = 0;
        int j = 0;
#pragma unroll 1
        for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, j++) {
            const int b = j & 1;
            if (j >= 2) {
                ok = __all_sync(0xffffffffu, mbar_wait(&acc_empty[b], (uint32_t)(((j >> 1) - 1) & 1)));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            const uint32_t d = tmem + (uint32_t)b * L::kAccCols;
#pragma unroll 1
            for (int kb = 0; kb < nk; kb++, g++) {
                const int s = g % S;
                ok = __all_sync(0xffffffffu, mbar_wait(&conv[s], (uint32_t)((g / S) & 1)));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t dh = dh0 + (uint64_t)((s * L::kStage) >> 4);
                const uint64_t dl = dh + (uint64_t)(L::kB >> 4);
                const uint32_t ahi = tmem + L::kACol0 + (uint32_t)(s * L::kACols);
                const uint32_t alo = ahi + kT3BK;
                if (leader) {
#pragma unroll
                    for (int k = 0; k < kT3BK / 8; k++) {
                        umma_tf32_ta(d, ahi + 8 * k, dh + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
                        umma_tf32_ta(d, ahi + 8 * k, dl + 2 * k, idesc, 1u);
                        umma_tf32_ta(d, alo + 8 * k, dh + 2 * k, idesc, 1u);
                    }
                    umma_commit(&empty[s]);
                }
                __syncwarp();
            }
            if (!ok) break;
            if (leader) umma_commit(&acc_full[b]);
            __syncwarp();
        }
        if (leader) {
            if (!ok) atomicExch(&abort_flag, 1);
            umma_commit(mma_done);
        }
        __syncwarp();
    } else if (warp >= 6) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 of the
        // accumulator, stages them in its own rows of the staging tile and
        // stores them; the accumulator is released as soon as it is read
        const int q = warp % 4;
        int j = 0;
#pragma unroll 1
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, j++) {
            const int b = j & 1;
            if (!mbar_wait(&acc_full[b], (uint32_t)((j >> 1) & 1))) {
                atomicExch(&abort_flag, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tc_stage_tile<L::BN, true>(tmem + (uint32_t)b * L::kAccCols, q, lane, staging);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
            __syncwarp();
            tc_store_rows<L::BN, EPI>(32 * q, 32, lane, (t / tiles_n) * kTcBM, (t % tiles_n) * L::BN, M, N, bias,
                                      Cm, nullptr, staging, 1, nullptr, nullptr);
            __syncwarp();
        }
    }

    const bool finished = mbar_wait(mma_done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if ((!finished || abort_flag) && threadIdx.x == 0) {
        atomicExch(err, 1);
        // let the last loads of every stage land before the CTA leaves
        for (int g = issued - 1; g >= 0 && g >= issued - S; g--)
            mbar_wait(&full[g % S], (uint32_t)((g / S) & 1));
        if (!finished) mbar_wait(mma_done, 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::kTmemCols));
}

// ------------------------------------------ persistent BF16 / E4M3 GEMM
//
// The compression-size projections of the BF16 and FP8 forms without split
// K, the same way as k_gemm_t3_persist: one CTA per SM walks the 128 x 128
// output tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...; the TMA warp and
// the MMA warp stream K blocks across tile boundaries through one ring of
// stages (A and B both by TMA, 128-byte rows: 64 BF16 or 128 E4M3 of K);
// tile j accumulates in TMEM accumulator j % 2 while four epilogue warps
// drain the other one through a staging buffer of their own.  Each tile
// sees the MMA sequence and epilogue arithmetic of k_gemm_tc_bf16 with
// BN = 128, so the bits are the same.  Warps: 0 TMA, 1 MMA, 2-5 epilogue.
struct TcP {
    static constexpr int BN = 128;
    static constexpr int kA = kTcBM * 128;                       // 16 KB
    static constexpr int kB = BN * 128;                          // 16 KB
    static constexpr int kStage = kA + kB;
    static constexpr int kStages = 4;
    static constexpr int kStaging = kTcBM * BN * 4;              // 64 KB
    static constexpr uint32_t kAccCols = BN;
    static constexpr uint32_t kTmemCols = 2 * kAccCols;
    static constexpr int kBars = 2 * kStages + 4 + 1;            // full, empty; acc_full[2], acc_empty[2]; mma_done
    static constexpr size_t kBytes = 1024 + (size_t)kStages * kStage + kStaging + 8 * kBars + 16;
    static constexpr int kThreads = 192;
};

template <int EPI, int KIND>
__global__ void __launch_bounds__(TcP::kThreads, 1)
k_gemm_tc_persist(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const float* __restrict__ bias, float* __restrict__ Cm, __nv_bfloat16* __restrict__ out_bf16,
                  int M, int N, int K, int* __restrict__ err, const float* __restrict__ row_scale,
                  const float* __restrict__ col_scale) {
    using L = TcP;
    constexpr int S = L::kStages;
    constexpr int kElemK = KIND == kKindE4M3 ? 128 : kTcBK;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    float* staging = reinterpret_cast<float*>(smem + (size_t)S * L::kStage);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * L::kStage + L::kStaging);
    uint64_t* full = bars;
    uint64_t* empty = bars + S;
    uint64_t* acc_full = bars + 2 * S;
    uint64_t* acc_empty = bars + 2 * S + 2;
    uint64_t* mma_done = bars + 2 * S + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + L::kBars);
    __shared__ int abort_flag;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int tiles_n = (N + L::BN - 1) / L::BN;
    const int n_tiles = tiles_n * ((M + kTcBM - 1) / kTcBM);
    const int nk = K / kElemK;

    if (threadIdx.x == 0) {
        tma_prefetch_map(&tmA);
        tma_prefetch_map(&tmB);
        abort_flag = 0;
        for (int i = 0; i < S; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
        }
        mbar_init(mma_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(L::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    pdl_launch_next();
    pdl_wait_prev();

    int issued = 0;
    if (threadIdx.x == 0) {
        // TMA producer
        int g = 0;
#pragma unroll 1
        for (int t = blockIdx.x; t < n_tiles && !*(volatile int*)&abort_flag; t += gridDim.x) {
            const int m0 = (t / tiles_n) * kTcBM, n0 = (t % tiles_n) * L::BN;
#pragma unroll 1
            for (int kb = 0; kb < nk; kb++, g++) {
                const int s = g % S;
                if (g >= S && !mbar_wait(&empty[s], (uint32_t)(((g / S) - 1) & 1))) {
                    atomicExch(&abort_flag, 1);
                    break;
                }
                uint8_t* st = smem + (size_t)s * L::kStage;
                mbar_expect_tx(&full[s], L::kStage);
                tma_load_2d(&tmA, &full[s], st, kb * kElemK, m0);
                tma_load_2d(&tmB, &full[s], st + L::kA, kb * kElemK, n0);
                issued = g + 1;
            }
        }
    } else if (warp == 1) {
        // MMA issuer: tile j accumulates in accumulator j % 2, after the
        // epilogue has read that accumulator's previous tile (j - 2)
        constexpr uint32_t idesc = KIND == kKindE4M3 ? umma_idesc_e4m3(kTcBM, L::BN) : umma_idesc_bf16(kTcBM, L::BN);
        const bool leader = elect_one();
        const uint64_t da0 = umma_desc_sw128(smem_u32(smem));
        const uint64_t db0 = umma_desc_sw128(smem_u32(smem + L::kA));
        bool ok = true;
        int g = 0, j = 0;
#pragma unroll 1
        for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, j++) {
            const int b = j & 1;
            if (j >= 2) {
                ok = __all_sync(0xffffffffu, mbar_wait(&acc_empty[b], (uint32_t)(((j >> 1) - 1) & 1)));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            const uint32_t d = tmem + (uint32_t)b * L::kAccCols;
#pragma unroll 1
            for (int kb = 0; kb < nk; kb++, g++) {
                const int s = g % S;
                ok = __all_sync(0xffffffffu, mbar_wait(&full[s], (uint32_t)((g / S) & 1)));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint64_t so = (uint64_t)((s * L::kStage) >> 4);
                if (leader) {
#pragma unroll
                    for (int k = 0; k < 4; k++) {   // 32 bytes of K per instruction
                        if (KIND == kKindE4M3)
                            umma_e4m3(d, da0 + so + 2 * k, db0 + so + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
                        else
                            umma_bf16(d, da0 + so + 2 * k, db0 + so + 2 * k, idesc, (kb | k) != 0 ? 1u : 0u);
                    }
                    umma_commit(&empty[s]);
                }
                __syncwarp();
            }
            if (!ok) break;
            if (leader) umma_commit(&acc_full[b]);
            __syncwarp();
        }
        if (leader) {
            if (!ok) atomicExch(&abort_flag, 1);
            umma_commit(mma_done);
        }
        __syncwarp();
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31
        const int q = warp % 4;
        int j = 0;
#pragma unroll 1
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, j++) {
            const int b = j & 1;
            if (!mbar_wait(&acc_full[b], (uint32_t)((j >> 1) & 1))) {
                atomicExch(&abort_flag, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tc_stage_tile<L::BN, true>(tmem + (uint32_t)b * L::kAccCols, q, lane, staging);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
            __syncwarp();
            tc_store_rows<L::BN, EPI>(32 * q, 32, lane, (t / tiles_n) * kTcBM, (t % tiles_n) * L::BN, M, N, bias,
                                      Cm, out_bf16, staging, 1, row_scale, col_scale);
            __syncwarp();
        }
    }

    const bool finished = mbar_wait(mma_done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if ((!finished || abort_flag) && threadIdx.x == 0) {
        atomicExch(err, 1);
        for (int g = issued - 1; g >= 0 && g >= issued - S; g--)
            mbar_wait(&full[g % S], (uint32_t)((g / S) & 1));
        if (!finished) mbar_wait(mma_done, 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::kTmemCols));
}

}  // namespace boa
