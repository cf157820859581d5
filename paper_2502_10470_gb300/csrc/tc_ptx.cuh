// tc_ptx.cuh -- inline-PTX building blocks of the tensor-core kernels
// (tc_rotate.cu, tc_fused.cu): mbarriers with bounded waits, 2-D TMA loads,
// tcgen05 MMA issue / commit / TMEM loads, the UMMA shared-memory and
// instruction descriptors, and the composition of objective states of
// consecutive column ranges.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "block.cuh"

namespace metade {
namespace tc {

constexpr int kBM = 128, kBN = 256, kBK = 64;           // BF16: a 64-element K tile is one 128-byte row
constexpr int kBK8 = 128;                                 // FP8: a 128-element K tile is one 128-byte row
constexpr float kE4M3Max = 448.0f;                        // largest finite e4m3 value
constexpr int kStages = 4;                                 // 4 stages (193 KB): one CTA per SM
constexpr int kParts = 4;                                  // epilogue warps per TMEM lane quadrant
constexpr int kEpiWarps = 4 * kParts;                      // each takes kBN / kParts columns of a chunk
constexpr int kTcThreads = 32 * (kEpiWarps + 1);           // + the producer/MMA warp
constexpr int kAT = kBM * kBK * 2;                        // 16 KB
constexpr int kBT = kBN * kBK * 2;                        // 32 KB
constexpr uint32_t kWaitLimit = 1u << 18;                 // try_wait rounds before giving up: ~1 s (a round waits <= 3.8 us)
constexpr int kStatusTimeout = 4;                         // METADE_ETIMEOUT

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t rounds = kWaitLimit) {
    const uint32_t addr = smem_u32(bar);
    for (uint32_t it = 0; it < rounds; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128
// bytes grouped by 8 (stride 1024 bytes), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: 8 rows x 128 bytes
    d |= (uint64_t)1 << 46;             // version
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: BF16 A and B, FP32 D, K-major, M 128, N 256.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

// Instruction descriptor, kind::f8f6f4: e4m3 A and B (format 0), FP32 D, K-major, M 128, N 256.
constexpr uint32_t kIdesc8 = (1u << 4) | ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);

// K 32 e4m3 elements per instruction: 32 bytes along the swizzled row, like BF16.
__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc8), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// a <- a followed by b, where b is the objective state of the next columns
// evaluated from a fresh state: zf is b's first z, q1 the sum of b's running
// prefixes (Schwefel 1.2) and nb its number of columns.
__device__ __forceinline__ void obj_compose(int obj, ObjR& a, const ObjR& b, float zf, float q1, int nb) {
    if (nb == 0) return;
    switch (obj) {
    case kAckley:
        a.s0 += b.s0;
        a.s1 += b.s1;
        break;
    case kGriewank:  // 1 - prod c over both: s1 = s1_a + prod_a s1_b
        a.s0 += b.s0;
        a.s1 = fmaf(a.pre, b.s1, a.s1);
        a.pre *= b.pre;
        break;
    case kRosenbrock:  // the pair across the boundary, then b's own pairs
        if (!a.first) {
            const float t = zf - a.prev * (a.prev + 2.f);
            a.s0 += 100.f * t * t + a.prev * a.prev;
        }
        a.s0 += b.s0;
        a.prev = b.prev;
        a.first = false;
        break;
    case kSchwefel12: {  // sum over b of (P + q_i)^2, P = a's prefix
        const float P = a.prev;
        a.s0 += b.s0 + (float)nb * P * P + 2.f * P * q1;
        a.prev = P + b.prev;
        break;
    }
    default: a.s0 += b.s0; break;
    }
}

}  // namespace tc
}  // namespace metade
