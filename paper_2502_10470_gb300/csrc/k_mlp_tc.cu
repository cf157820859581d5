// k_mlp_tc.cu -- the MLP objective's evaluation on the tensor cores, for
// contexts whose precision is BF16 or bf16x3.
//
// An individual's first layer is a small dense GEMM, Z1 [256 inputs][h] =
// X [256][16] . W1 [16][h]: M 256 (two 128-row tiles), K 16 (one MMA), N = h
// rounded up to 16 (the instruction's N).  X is the same for every individual
// and stays in shared memory; W1 differs per individual.  k_mlp_tc is
// persistent (two CTAs of 256 threads per SM, TMEM 256 columns each: one
// CTA's loads overlap the other's epilogue) and walks its individuals:
//   load      the trial row (all 19 h + 2 parameters) into a shared buffer,
//             then W1^T as the B operand (BF16 hi, and lo = bf16(w - hi) for
//             bf16x3), K-major with the 128-byte swizzle the UMMA descriptor
//             reads; the K columns past 16 are never read (one K-16 step)
//   MMA       thread 0 issues tcgen05.mma (M 128, N h_pad, K 16; bf16x3:
//             hi.hi, hi.lo, lo.hi into one accumulator) for both M tiles into
//             two TMEM accumulators and commits to an mbarrier
//   epilogue  thread = input (warp w
//             reads TMEM lanes 32 (w % 4).. of M tile w / 4), tanh(z + b1)
//             (the hardware tanh.approx in BF16, tanhf in bf16x3), the second
//             layer in FP32 as two interleaved chains per output (even and odd
//             hidden units) plus the output bias, the squared error against
//             the teacher, a block sum in warp order
// so the differences from the FP32 kernel are the operands' rounding, the
// BF16 context's tanh, and the order of the sums.  Every mbarrier wait is
// bounded; on timeout the kernel latches METADE_ETIMEOUT, waits (bounded) for
// its own MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include "block.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace metade {

namespace {

using namespace tc;

constexpr int kMTThreads = 256;            // 8 warps: (M tile, TMEM lane quadrant)
constexpr int kMTAcc = 128;                // TMEM columns per accumulator (h_pad <= 80 used)
constexpr int kMTRows = 128;               // rows of a 128-byte-swizzled operand tile
constexpr size_t kMTTile = (size_t)kMTRows * 128;  // bytes of one operand tile (16 KB)
constexpr int kMTMaxDpad = 1536;           // floats of a staged parameter row

// Byte offset of K byte `kb` of row `row` in a K-major tile with the 128-byte
// swizzle: 8-row atoms of 1024 bytes, 16-byte chunk c of row r stored at chunk c ^ (r % 8).
__device__ __forceinline__ uint32_t sw128_off(int row, int kb) {
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((kb >> 4) ^ (row & 7)) << 4) | (kb & 15)));
}

__device__ __forceinline__ uint32_t bf16_bits(float x) {
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    return (uint32_t)*reinterpret_cast<const unsigned short*>(&b);
}

// Elements (row, k) and (row, k + 1) as hi BF16 (and lo = bf16(x - hi)) into the tiles.
__device__ __forceinline__ void put_pair(uint8_t* hi, uint8_t* lo, int row, int k, float x0, float x1) {
    const uint32_t h0 = bf16_bits(x0), h1 = bf16_bits(x1);
    const uint32_t off = sw128_off(row, 2 * k);
    *reinterpret_cast<uint32_t*>(hi + off) = h0 | (h1 << 16);
    if (lo) {
        const float r0 = x0 - __uint_as_float(h0 << 16), r1 = x1 - __uint_as_float(h1 << 16);
        *reinterpret_cast<uint32_t*>(lo + off) = bf16_bits(r0) | (bf16_bits(r1) << 16);
    }
}

__device__ __forceinline__ void mma_bf16_n(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// tanh of the hidden layer: the hardware approximation (tanh.approx.f32, relative
// error about 2^-11, below BF16's operand rounding) in BF16; tanhf in bf16x3
__device__ __forceinline__ float act(float x, bool accurate) {
    if (accurate) return tanhf(x);
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct MlpTcArgs {
    const InstDesc* desc;
    const int* row_exec;   // row -> executor (InstDesc.tc_row = its first row)
    int n_rows;
    const float* rows;     // parameter rows (population layout)
    const float* x;        // inputs [256][16]
    const float* y;        // teacher outputs ([256][2] at InstDesc.aux)
    float* f_out;          // fitness layout
    int split;             // 1: bf16x3
    int* status;
};

__global__ void __launch_bounds__(kMTThreads, 2) k_mlp_tc(MlpTcArgs g) {
    extern __shared__ uint8_t smraw[];
    __shared__ __align__(8) uint64_t mbar, drain;
    __shared__ uint32_t tmem_base;
    __shared__ float part[kMTThreads / 32];
    __shared__ int abort_s;
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    uint8_t* Ahi = sm;                       // 2 M tiles: inputs 0..127, 128..255
    uint8_t* Bhi = Ahi + 2 * kMTTile;        // W1^T of the individual
    float* prow = reinterpret_cast<float*>(Bhi + kMTTile);  // [kMTMaxDpad] its parameter row
    uint8_t* Alo = reinterpret_cast<uint8_t*>(prow + kMTMaxDpad);  // bf16x3 only
    uint8_t* Blo = Alo + 2 * kMTTile;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool split = g.split != 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * kMTAcc)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&mbar, 1);
        mbar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    // the inputs as the A operand, both M tiles
    for (int e = tid; e < kMlpN * (kMlpIn / 2); e += kMTThreads) {
        const int n = e / (kMlpIn / 2), k = 2 * (e - n * (kMlpIn / 2));
        const int m = n / kMTRows, row = n - m * kMTRows;
        put_pair(Ahi + m * kMTTile, split ? Alo + m * kMTTile : nullptr, row, k, g.x[n * kMlpIn + k],
                 g.x[n * kMlpIn + k + 1]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tmem_base;

    const int m = warp >> 2, q = warp & 3;      // epilogue: M tile, TMEM lane quadrant
    const int n = m * kMTRows + q * 32 + lane;  // this thread's input
    bool mma_any = false;
    int j = 0;
    for (int r = blockIdx.x; r < g.n_rows; r += gridDim.x, ++j) {
        const InstDesc d = g.desc[g.row_exec[r]];
        const float* u = g.rows + d.pop_off + (long long)(r - d.tc_row) * d.dpad;
        for (int e = tid; e < d.dpad / 4; e += kMTThreads)
            reinterpret_cast<float4*>(prow)[e] = __ldg(reinterpret_cast<const float4*>(u) + e);
        __syncthreads();
        const int h = mlp_hidden(d.dim);
        const int hpad = (h + 15) & ~15;
        for (int e = tid; e < hpad * (kMlpIn / 2); e += kMTThreads) {  // W1^T: row jr, K k, k + 1 (zero rows past h)
            const int jr = e / (kMlpIn / 2), k = 2 * (e - jr * (kMlpIn / 2));
            const float w0 = jr < h ? prow[k * h + jr] : 0.f, w1 = jr < h ? prow[(k + 1) * h + jr] : 0.f;
            put_pair(Bhi, split ? Blo : nullptr, jr, k, w0, w1);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {  // the individual's MMAs into accumulators 0 and 1 (M tiles)
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(hpad >> 3) << 17) |
                                   ((uint32_t)(kMTRows >> 4) << 24);
            const uint64_t bh = sdesc_sw128(smem_u32(Bhi));
            const uint64_t bl = sdesc_sw128(smem_u32(Blo));
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const uint32_t dt = taddr + (uint32_t)(mt * kMTAcc);
                const uint64_t ah = sdesc_sw128(smem_u32(Ahi + mt * kMTTile));
                mma_bf16_n(dt, ah, bh, idesc, 0u);
                if (split) {
                    const uint64_t al = sdesc_sw128(smem_u32(Alo + mt * kMTTile));
                    mma_bf16_n(dt, ah, bl, idesc, 1u);
                    mma_bf16_n(dt, al, bh, idesc, 1u);
                }
            }
            mma_commit(&mbar);
            mma_any = true;
        }
        const float* b1 = prow + kMlpIn * h;
        const float* W2 = b1 + h;
        const float* b2 = W2 + kMlpOut * h;
        const bool got = __all_sync(kFull, mbar_wait(&mbar, (uint32_t)(j & 1)) ? 1 : 0) != 0;
        tc_fence_after();
        float e2 = 0.f;
        if (got) {
            // the second layer in two interleaved chains per output (even and odd j), added at the end
            float y0a = 0.f, y0b = 0.f, y1a = 0.f, y1b = 0.f;
            const uint32_t base = taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)(m * kMTAcc);
            for (int c0 = 0; c0 < h; c0 += 32) {  // uniform over the warp
                float v[32];
                tmem_ld32(base + (uint32_t)c0, v);
#pragma unroll
                for (int c = 0; c < 32; c += 2) {
                    if (c0 + c < h) {
                        const float t = act(v[c] + b1[c0 + c], split);
                        y0a = fmaf(t, W2[2 * (c0 + c)], y0a);
                        y1a = fmaf(t, W2[2 * (c0 + c) + 1], y1a);
                    }
                    if (c0 + c + 1 < h) {
                        const float t = act(v[c + 1] + b1[c0 + c + 1], split);
                        y0b = fmaf(t, W2[2 * (c0 + c + 1)], y0b);
                        y1b = fmaf(t, W2[2 * (c0 + c + 1) + 1], y1b);
                    }
                }
            }
            const float y0 = b2[0] + (y0a + y0b), y1 = b2[1] + (y1a + y1b);
            const float d0 = y0 - g.y[d.aux + 2 * n], d1 = y1 - g.y[d.aux + 2 * n + 1];
            e2 = fmaf(d0, d0, d1 * d1);
        } else if (lane == 0) {
            set_status(g.status, kStatusTimeout);
            abort_s = 1;
        }
        tc_fence_before();
        const float s = warp_sum(e2);
        if (lane == 0) part[warp] = s;
        __syncthreads();  // also: prow, B and the accumulators are free for the next individual
        if (tid == 0 && !abort_s) {
            float t = 0.f;
            for (int w = 0; w < kMTThreads / 32; ++w) t += part[w];
            g.f_out[d.fit_off + (r - d.tc_row)] = nan_to_inf(t * (1.0f / (kMlpN * kMlpOut)));
        }
        if (abort_s) break;  // uniform: read after the barrier
    }
    if (tid == 0 && mma_any) {  // no MMA of this CTA in flight when TMEM is freed (bounded)
        mma_commit(&drain);
        mbar_wait(&drain, 0u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(2 * kMTAcc) : "memory");
}

// A, B and the parameter row; the lo tiles too for bf16x3
size_t mlp_tc_smem(bool split) {
    return 1024 + 3 * kMTTile + (size_t)kMTMaxDpad * sizeof(float) + (split ? 3 * kMTTile : 0);
}

}  // namespace

cudaError_t launch_mlp_eval_tc(const InstDesc* desc, const MlpPlan& p, const float* rows, float* f_out, int* status,
                               cudaStream_t st) {
    if (p.n_rows <= 0) return cudaSuccess;
    const size_t smem = mlp_tc_smem(p.tc == 2);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    MlpTcArgs g;
    g.desc = desc;
    g.row_exec = p.row_exec;
    g.n_rows = p.n_rows;
    g.rows = rows;
    g.x = p.x;
    g.y = p.y;
    g.f_out = f_out;
    g.split = p.tc == 2 ? 1 : 0;
    g.status = status;
    const int grid = p.n_rows < 2 * p.sms ? p.n_rows : 2 * p.sms;  // two CTAs per SM (TMEM 256 columns each)
    k_mlp_tc<<<grid, kMTThreads, smem, st>>>(g);
    return cudaGetLastError();
}

}  // namespace metade
