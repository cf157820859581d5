// tc_rotate.cu -- large-D executors on the 5th-generation tensor cores.
//
// For D >= 256 the rotation z = R (u - o) of a whole population is a dense
// GEMM, Z[NP x D] = Dq[NP x K] * Rq[D x K]^T, with both operands K-major.  One
// generation of the large-D executors is four launches:
//   k_tc_prologue  best and pbest pool per executor (block per executor)
//   k_tc_trial     draws, mutation, crossover, clip (warp per individual);
//                  writes the FP32 trial row and the BF16 GEMM operand(s)
//   k_rot_tc       tcgen05 GEMM: TMA (128-byte swizzle, 4 stages) -> shared
//                  memory -> tcgen05.mma (M 128, N 256, K 16, FP32 accumulate
//                  into one of two TMEM accumulators) issued by a producer
//                  warp; four epilogue warps read TMEM with tcgen05.ld, one
//                  thread per individual (TMEM lane), and accumulate the
//                  objective column chunk by column chunk while the MMAs of
//                  the next chunk run, so Z never reaches memory
//   k_tc_select    greedy selection and row copy (warp per individual);
//                  near ties are listed for k_tc_ties (a CTA per tie)
// Precision: BF16 operands, or bf16x3 (split precision, Henry, Tang &
// Heinecke, ARITH 2019): d = d_hi + d_lo, R = R_hi + R_lo, and
// Z = d_hi R_hi + d_hi R_lo + d_lo R_hi accumulated in FP32.
//
// Every mbarrier wait is bounded: on timeout the kernel latches
// METADE_ETIMEOUT, drains its own outstanding copies (bounded), frees TMEM
// and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "block.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace metade {

namespace {

using namespace tc;

// The bounded wait on its own: one thread initialises an mbarrier for one
// arrival, arrives on it first when `arrive` is set, and waits on phase 0 for
// at most `rounds` try_wait rounds (every wait of the GEMM pipeline is this
// loop with kWaitLimit rounds).  out[0] = 1 when the phase completed, else the
// timeout is latched in *status; out[1] = the SM clock cycles the wait took.
__global__ void k_wait_check(uint32_t rounds, int arrive, long long* out, int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
    const long long t0 = clock64();
    const bool done = mbar_wait(&bar, 0u, rounds);
    out[1] = clock64() - t0;
    out[0] = done ? 1 : 0;
    if (!done) set_status(status, kStatusTimeout);
}

struct TcGemmArgs {
    const InstDesc* desc;
    const int* tiles;         // [n_tiles][2]: first operand row of the tile, rows (<= 128), all of one problem
    const int* row_exec;      // operand row -> executor
    const long long* brow;    // per problem: first row of its padded R in the B operand
    float* fu;                // out: f(u) per individual (fitness index)
    int kt;                   // K tiles (128 bytes: 64 BF16 or 128 e4m3 elements)
    int split;                // 1: bf16x3 (three products)
    int fp8;                  // 1: e4m3 operands, z = acc * ascale[row] * bscale[problem]
    const float* ascale;      // FP8: per operand row, max|d| / 448
    const float* bscale;      // FP8: per problem, max|R| / 448
    int* status;
    // selection in the epilogue (sel = 1, BF16 with FP32-difference ties): the row's decision
    // against the stored fitness, clear acceptances committed, near ties listed for k_tc_ties2
    int sel;
    float* pop;               // population (rows committed here)
    float* fit;               // stored fitness
    const float* uscr;        // trial rows
    const float* theta;       // decoded theta per executor (rows of an invalid theta are left alone)
    const int* prob_tp;       // problem -> index among the problems on the path
    const int* tp_row0;       // per such problem: start of its tie list
    int* tie_cnt;             // per such problem: near ties listed
    int* tie_list;            // fitness index of each near tie
    long long* tie_off;       // population offset of each near tie's row
};

// kTcThreads threads.  Warps 0 .. kEpiWarps-1 run the epilogue: warp w reads
// TMEM lanes 32 (w % 4).. (tile rows) and column part w / 4 (kBN / kParts
// columns) of every chunk; parts 1.. start from a fresh objective state and
// hand it over through shared memory (part_ready) to part 0, which composes
// them in column order.  Lane 0 of the last warp issues the TMA loads and the
// MMAs.  Two accumulators of kBN TMEM columns: the MMAs of
// column chunk c + 1 run while the epilogue drains chunk c (acc_full: the
// chunk's MMAs are done; acc_empty: the four epilogue warps have read it).
__global__ void __launch_bounds__(kTcThreads, 1)
    k_rot_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
             const __grid_constant__ CUtensorMap tmAlo, const __grid_constant__ CUtensorMap tmBlo, TcGemmArgs a) {
    extern __shared__ uint8_t smraw[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2], part_ready[4][2], drain;
    __shared__ __align__(16) float part[2][kParts - 1][kBM][8];
    __shared__ uint32_t tmem_base;
    __shared__ int nacc_s;
    __shared__ long long acc_off[kBM];  // selection mode: population offsets of the accepted rows
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    const int nops = a.split ? 2 : 1;  // operand sets per stage (hi, and lo when split)
    const int stage_bytes = nops * (kAT + kBT);
    const int nst = a.split ? 2 : kStages;  // pipeline depth that fits shared memory
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int arow = a.tiles[2 * blockIdx.x], nr = a.tiles[2 * blockIdx.x + 1];  // first operand row, rows
    const InstDesc d = a.desc[a.row_exec[arow]];  // dim, objective and problem are those of every row of the tile
    const int brow0 = (int)a.brow[d.prob];
    const int nchunks = (d.dim + kBN - 1) / kBN;
    const int kel = a.fp8 ? kBK8 : kBK;  // K elements per 128-byte tile (x is in elements, 128 bytes apart)
    // K tiles of this tile's problem: operand columns past its D_pad are zero (or not written)
    const int kt = min(a.kt, (d.dpad + kel - 1) / kel);
    const int total = nchunks * kt;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * kBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpiWarps);  // one arrival per epilogue warp
            for (int q = 0; q < 4; ++q) mbar_init(&part_ready[q][b], kParts - 1);
        }
        mbar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        nacc_s = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tmem_base;

    auto load = [&](int it) {
        const int s = it % nst, c = it / kt, kk = it - c * kt;
        uint8_t* st = sm + s * stage_bytes;
        mbar_expect_tx(&full[s], (uint32_t)stage_bytes);
        tma_load_2d(st, &tmA, &full[s], kk * kel, arow);
        tma_load_2d(st + kAT, &tmB, &full[s], kk * kel, brow0 + c * kBN);
        if (a.split) {
            tma_load_2d(st + kAT + kBT, &tmAlo, &full[s], kk * kel, arow);
            tma_load_2d(st + 2 * kAT + kBT, &tmBlo, &full[s], kk * kel, brow0 + c * kBN);
        }
    };

    if (warp == kEpiWarps) {
        if (lane == 0) {
            bool ok = true;
            int issued = 0, consumed = 0;  // loads issued / waited on
            const int pre = total < nst ? total : nst;
            for (int it = 0; it < pre; ++it) load(it);
            issued = pre;
            for (int c = 0; c < nchunks && ok; ++c) {
                const int b = c & 1;
                const uint32_t dacc = taddr + (uint32_t)(b * kBN);
                // the epilogue has drained this accumulator (chunk c - 2)
                if (c >= 2 && !mbar_wait(&acc_empty[b], (uint32_t)((c - 2) >> 1) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int kk = 0; kk < kt; ++kk) {
                    const int it = c * kt + kk, s = it % nst;
                    if (!mbar_wait(&full[s], (uint32_t)(it / nst) & 1u)) {
                        ok = false;
                        break;
                    }
                    ++consumed;
                    tc_fence_after();
                    uint8_t* st = sm + s * stage_bytes;
                    const uint64_t ad = sdesc_sw128(smem_u32(st)), bd = sdesc_sw128(smem_u32(st + kAT));
                    if (a.fp8) {
#pragma unroll
                        for (int j = 0; j < 4; ++j)  // K 32 per instruction, 32 bytes along the swizzled row
                            mma_e4m3(dacc, ad + 2 * j, bd + 2 * j, (kk > 0 || j > 0) ? 1u : 0u);
                    } else {
#pragma unroll
                        for (int j = 0; j < kBK / 16; ++j)  // K 16 per instruction, 32 bytes along the swizzled row
                            mma_bf16(dacc, ad + 2 * j, bd + 2 * j, (kk > 0 || j > 0) ? 1u : 0u);
                    }
                    if (a.split) {
                        const uint64_t al = sdesc_sw128(smem_u32(st + kAT + kBT));
                        const uint64_t bl = sdesc_sw128(smem_u32(st + 2 * kAT + kBT));
#pragma unroll
                        for (int j = 0; j < kBK / 16; ++j) {
                            mma_bf16(dacc, ad + 2 * j, bl + 2 * j, 1u);
                            mma_bf16(dacc, al + 2 * j, bd + 2 * j, 1u);
                        }
                    }
                    mma_commit(&empty[s]);
                    // refill the stage used by the previous iteration once its MMAs are done
                    if (it >= 1 && issued < total) {
                        const int pit = it - 1, ps = pit % nst;
                        if (!mbar_wait(&empty[ps], (uint32_t)(pit / nst) & 1u)) {
                            ok = false;
                            break;
                        }
                        load(issued);
                        ++issued;
                    }
                }
                if (ok) mma_commit(&acc_full[b]);
            }
            if (!ok) {
                set_status(a.status, kStatusTimeout);
                // drain copies still in flight into this CTA's shared memory (bounded)
                for (int it = consumed; it < issued; ++it) mbar_wait(&full[it % nst], (uint32_t)(it / nst) & 1u);
                // and every MMA already issued: a commit tracks all of this thread's earlier tcgen05
                // operations, so once `drain` completes (bounded) none still writes TMEM or reads
                // shared memory when the CTA frees them
                mma_commit(&drain);
                mbar_wait(&drain, 0u);
            }
        }
        __syncwarp();
    } else {
        const int qd = warp & 3, half = warp >> 2;  // half: this warp's column part of every chunk
        constexpr int kBpp = kBN / 32 / kParts;       // 32-column blocks per part
        ObjR acc;                           // part 0: the row's running state; parts 1..: the chunk's
        const int row = 32 * qd + lane;     // tile row of this thread
        // FP8: dequantisation factor of this row (rows past the executor are not used)
        const float zs = (a.fp8 && row < nr) ? a.ascale[arow + row] * a.bscale[d.prob] : 1.0f;
        // selection mode: the row's executor fields and stored fitness, fetched before the chunks so that
        // these dependent loads overlap the epilogue's work
        bool rok = false;
        int fidx = 0;
        long long roff = 0;
        float fx = 0.f;
        if (a.sel && half == 0 && row < nr) {
            const int k = a.row_exec[arow + row];
            const InstDesc e = a.desc[k];
            rok = load_strat(a.theta + 6 * k, e.np).ok;  // rows of an invalid theta are left alone
            fidx = e.fit_off + (arow + row - e.tc_row);
            roff = e.pop_off + (long long)(arow + row - e.tc_row) * d.dpad;
            if (rok) fx = a.fit[fidx];
        }
        bool eok = true;
        for (int c = 0; c < nchunks; ++c) {
            const int b = c & 1;
            const bool got = __all_sync(kFull, mbar_wait(&acc_full[b], (uint32_t)(c >> 1) & 1u) ? 1 : 0) != 0;
            if (!got) {
                eok = false;
                break;
            }
            tc_fence_after();
            if (half) acc = ObjR();          // parts 1..: this chunk's columns from a fresh state
            float zf = 0.f, q1 = 0.f, qrun = 0.f;
            int nb = 0;
            for (int p = kBpp * half; p < kBpp * (half + 1); ++p) {
                const int col0 = c * kBN + 32 * p;
                if (col0 >= d.dim) break;  // uniform across the warp
                float v[32];
                tmem_ld32(taddr + ((uint32_t)(32 * qd) << 16) + (uint32_t)(b * kBN + 32 * p), v);
                if (a.fp8) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] *= zs;
                }
                if (half) {
                    if (nb == 0) zf = v[0];
                    const int m = min(32, d.dim - col0);
                    if (d.obj == kSchwefel12) {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j < m) {
                                qrun += v[j];
                                q1 += qrun;
                            }
                    }
                    nb += m;
                }
                acc.push32(d.obj, v, col0, d.dim);
            }
            tc_fence_before();
            __syncwarp();
            if (half) {
                float* sl = part[b][half - 1][row];
                *reinterpret_cast<float4*>(sl) = make_float4(acc.s0, acc.s1, acc.prev, acc.pre);
                *reinterpret_cast<float4*>(sl + 4) = make_float4(zf, q1, __int_as_float(nb), 0.f);
                __syncwarp();
                if (lane == 0) {
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&part_ready[qd][b])) : "memory");
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
                }
            } else {
                const bool have = __all_sync(kFull, mbar_wait(&part_ready[qd][b], (uint32_t)(c >> 1) & 1u) ? 1 : 0) != 0;
                if (!have) {
                    eok = false;
                    break;
                }
                for (int j = 0; j < kParts - 1; ++j) {
                    const float* sl = part[b][j][row];
                    const float4 x0 = *reinterpret_cast<const float4*>(sl), x1 = *reinterpret_cast<const float4*>(sl + 4);
                    ObjR rb;
                    rb.s0 = x0.x;
                    rb.s1 = x0.y;
                    rb.prev = x0.z;
                    rb.pre = x0.w;
                    rb.first = __float_as_int(x1.z) == 0;
                    obj_compose(d.obj, acc, rb, x1.x, x1.y, __float_as_int(x1.z));
                }
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
            }
        }
        if (!eok) {
            if (lane == 0) set_status(a.status, kStatusTimeout);
        } else if (half == 0 && row < nr) {
            const float fn = nan_to_inf(acc.finish(d.obj, d.dim));
            if (!a.sel) {
                const int k = a.row_exec[arow + row];
                const InstDesc& e = a.desc[k];  // this row's executor
                a.fu[e.fit_off + (arow + row - e.tc_row)] = fn;
            } else if (rok) {
                if (near_tie(fn, fx, tie_band(d.dim))) {
                    const int tp = a.prob_tp[d.prob];
                    const int q = a.tp_row0[tp] + atomicAdd(&a.tie_cnt[tp], 1);
                    a.tie_list[q] = fidx;
                    a.tie_off[q] = roff;
                } else if (fn <= fx) {
                    acc_off[atomicAdd(&nacc_s, 1)] = roff;
                    a.fit[fidx] = fn;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (a.sel) {  // accepted rows into the population, every thread copying float4s
        const int f4 = d.dpad >> 2, n = nacc_s * f4;
        for (int e2 = tid; e2 < n; e2 += blockDim.x) {
            const int q = e2 / f4, c4 = e2 - q * f4;
            const long long off = acc_off[q] + 4 * c4;
            *reinterpret_cast<float4*>(a.pop + off) = *reinterpret_cast<const float4*>(a.uscr + off);
        }
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(2 * kBN) : "memory");
}

// ----------------------------------------------------------- other stages
// One operand row of kp elements from v[0..dim) (zero past dim), by a warp.
// BF16: hi = bf16(v), and lo = bf16(v - hi) when split.  FP8: a per-row scale
// maps max|v| to 448, q = e4m3(v * scale) (round to nearest, saturating), and
// max|v| / 448 goes to *inv_scale for the GEMM epilogue.
__device__ __forceinline__ void pack_operand_row(const float* v, int dim, int kp, void* q, void* q_lo, long long r,
                                                 int fp8, float* inv_scale) {
    if (!q) return;  // FP32 GEMM on the CUDA cores: no operand rows
    const int lane = threadIdx.x & 31;
    if (fp8) {
        float m = 0.0f;
        for (int j = lane; j < dim; j += 32) m = fmaxf(m, fabsf(v[j]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
        const float sc = m > 0.0f ? kE4M3Max / m : 1.0f;
        if (lane == 0) *inv_scale = m > 0.0f ? m / kE4M3Max : 1.0f;
        uint8_t* row = reinterpret_cast<uint8_t*>(q) + r * kp;
        for (int j = lane; j < kp; j += 32)
            row[j] = j < dim ? (uint8_t)__nv_cvt_float_to_fp8(v[j] * sc, __NV_SATFINITE, __NV_E4M3) : (uint8_t)0;
        return;
    }
    // four elements per lane and step (kp is a multiple of 64, v holds round_up(dim, 4) floats)
    __nv_bfloat16* row = reinterpret_cast<__nv_bfloat16*>(q) + r * kp;
    __nv_bfloat16* row_lo = q_lo ? reinterpret_cast<__nv_bfloat16*>(q_lo) + r * kp : nullptr;
    for (int j = 4 * lane; j < kp; j += 128) {
        float x[4];
        if (j < dim) {
            const float4 x4 = *reinterpret_cast<const float4*>(v + j);
            x[0] = x4.x;
            x[1] = j + 1 < dim ? x4.y : 0.0f;
            x[2] = j + 2 < dim ? x4.z : 0.0f;
            x[3] = j + 3 < dim ? x4.w : 0.0f;
        } else {
            x[0] = x[1] = x[2] = x[3] = 0.0f;
        }
        const __nv_bfloat162 h01 = __floats2bfloat162_rn(x[0], x[1]), h23 = __floats2bfloat162_rn(x[2], x[3]);
        *reinterpret_cast<uint2*>(row + j) = make_uint2(*reinterpret_cast<const uint32_t*>(&h01),
                                                        *reinterpret_cast<const uint32_t*>(&h23));
        if (row_lo) {  // lo = bf16(x - hi)
            const __nv_bfloat162 l01 = __floats2bfloat162_rn(x[0] - __low2float(h01), x[1] - __high2float(h01));
            const __nv_bfloat162 l23 = __floats2bfloat162_rn(x[2] - __low2float(h23), x[3] - __high2float(h23));
            *reinterpret_cast<uint2*>(row_lo + j) = make_uint2(*reinterpret_cast<const uint32_t*>(&l01),
                                                               *reinterpret_cast<const uint32_t*>(&l23));
        }
    }
}

// Four BF16 operand elements at row[j..j+3] (8-byte aligned), and their lo
// residuals bf16(x - hi) at row_lo when it is set.
__device__ __forceinline__ void store_bf16x4(__nv_bfloat16* row, __nv_bfloat16* row_lo, int j, const float (&x)[4]) {
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(x[0], x[1]), h23 = __floats2bfloat162_rn(x[2], x[3]);
    *reinterpret_cast<uint2*>(row + j) = make_uint2(*reinterpret_cast<const uint32_t*>(&h01),
                                                    *reinterpret_cast<const uint32_t*>(&h23));
    if (row_lo) {
        const __nv_bfloat162 l01 = __floats2bfloat162_rn(x[0] - __low2float(h01), x[1] - __high2float(h01));
        const __nv_bfloat162 l23 = __floats2bfloat162_rn(x[2] - __low2float(h23), x[3] - __high2float(h23));
        *reinterpret_cast<uint2*>(row_lo + j) = make_uint2(*reinterpret_cast<const uint32_t*>(&l01),
                                                           *reinterpret_cast<const uint32_t*>(&l23));
    }
}

// Best and pbest pool from the generation-start fitness (block per executor).
__global__ void k_tc_prologue(StepArgs a, const int* __restrict__ execs, int* topk_all) {
    const int k = execs[blockIdx.x];
    const InstDesc d = a.desc[k];
    const Strat s = load_strat(a.theta + 6 * k, d.np);
    if (!s.ok) {
        if (threadIdx.x == 0) set_status(a.status, 1);
        return;
    }
    block_topk_staged(a.fit + d.fit_off, d.np, d.kp, topk_all + d.fit_off);
}

// Trial rows (FP32, into the scratch U) and the GEMM operand d = u - o: BF16
// (hi, and lo = bf16(d - hi) when split) or e4m3 with a per-row scale, K
// zero-padded to kp elements.
// Warps of one block may belong to different executors: per-warp shared
// scratch is strided by the bucket's widest row (ws floats).
__global__ void __launch_bounds__(256, 3) k_tc_trial(StepArgs a, const int* __restrict__ row_exec, int n_rows,
                                                  const int* __restrict__ topk_all, float* uscr, void* aq, void* aq_lo,
                                                  int kp, int ws, int fp8, float* ascale) {
    extern __shared__ __align__(16) float smt[];
    const int warp = threadIdx.x >> 5;
    const int r = blockIdx.x * (blockDim.x >> 5) + warp;
    if (r >= n_rows) return;
    const int k = row_exec[r];
    const InstDesc d = a.desc[k];
    const int i = r - d.tc_row;
    const Strat s = load_strat(a.theta + 6 * k, d.np);
    if (!s.ok) return;
    const uint32_t epoch = a.epoch_dev ? *a.epoch_dev : a.epoch;
    const Ctr c = make_ctr(a.key, (uint32_t)d.stream, a.gen0, (uint32_t)i, epoch);
    const int* topk = topk_all + d.fit_off;
    Indiv v;
    indiv_setup(s, c, i, d.np, d.dim, d.kp, topk, topk[0], v);
    const int L = s.cs == 2 ? warp_exp_length(c, d.dim, s.cri) : 0;  // uniform over the warp (one row)
    float* U = uscr + d.pop_off + (long long)i * d.dpad;
    // operand: none (FP32 GEMM on the CUDA cores), FP8 (the row's scale needs max |u - o| first, so u - o
    // is staged in shared memory, ws floats per warp), or BF16 packed by each lane as it builds its four
    // coordinates (hi, and lo = bf16(d - hi) when split).  One call site: the trial code is inlined once.
    const int mode = !aq ? 0 : (fp8 ? 1 : 2);
    float* db = smt + (size_t)warp * ws;
    __nv_bfloat16* row = mode == 2 ? reinterpret_cast<__nv_bfloat16*>(aq) + (long long)r * kp : nullptr;
    __nv_bfloat16* row_lo = mode == 2 && aq_lo ? reinterpret_cast<__nv_bfloat16*>(aq_lo) + (long long)r * kp : nullptr;
    warp_trial_to(s, c, v, i, d.dim, L, a.pop + d.pop_off, d.dpad, a.shift + d.shift_off, a.lo, a.hi, U,
                  [&](int j4, const float (&dd)[4]) {
                      if (mode == 2) store_bf16x4(row, row_lo, j4, dd);
                      else if (mode == 1) *reinterpret_cast<float4*>(db + j4) = make_float4(dd[0], dd[1], dd[2], dd[3]);
                  });
    if (mode == 1) {
        __syncwarp();
        pack_operand_row(db, d.dim, kp, aq, aq_lo, r, fp8, ascale + r);
    } else if (mode == 2) {
        const float zero[4] = {0.f, 0.f, 0.f, 0.f};
        for (int j = d.dpad + 4 * (threadIdx.x & 31); j < kp; j += 128) store_bf16x4(row, row_lo, j, zero);
    }
}

// Greedy selection and row copy.  Near ties are only listed here: with FP32
// difference-form ties per problem (fitness index and row offset, tl set) for
// the batched tie kernels, else in one list of operand rows for k_tc_ties,
// which decides each with a whole CTA (a warp alone would stream two D x D
// rotations from L2 one row group at a time).
__global__ void __launch_bounds__(256) k_tc_select(StepArgs a, const int* __restrict__ row_exec, int n_rows,
                                                   const float* __restrict__ uscr, const float* __restrict__ fu,
                                                   int* tie_list, int* tie_count, TieLists tl) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + warp;
    if (r >= n_rows) return;
    const int k = row_exec[r];
    const InstDesc d = a.desc[k];
    const Strat s = load_strat(a.theta + 6 * k, d.np);
    if (!s.ok) return;
    const int i = r - d.tc_row;
    float* X = a.pop + d.pop_off + (long long)i * d.dpad;
    const float* U = uscr + d.pop_off + (long long)i * d.dpad;
    float fn = fu[d.fit_off + i];
    const float fx = a.fit[d.fit_off + i];
    bool tie = near_tie(fn, fx, tie_band(d.dim));
    if (tie) {
        bool diff = false;
        for (int j = lane; j < d.dim; j += 32) diff = diff || (U[j] != X[j]);
        if (!__any_sync(kFull, diff)) tie = false, fn = fx;  // trial == target
    }
    if (tie) {
        if (lane == 0) {
            if (tl.tie_cnt) {  // per problem, for the batched tie kernels: fitness index and row offset
                const int tp = tl.prob_tp[d.prob];
                const int q = tl.tp_row0[tp] + atomicAdd(&tl.tie_cnt[tp], 1);
                tie_list[q] = d.fit_off + i;
                tl.tie_off[q] = d.pop_off + (long long)i * d.dpad;
            } else {
                tie_list[atomicAdd(tie_count, 1)] = r;
            }
        }
        return;
    }
    if (fn <= fx) {
        for (int j = lane * 4; j < d.dpad; j += 128)
            *reinterpret_cast<float4*>(X + j) = *reinterpret_cast<const float4*>(U + j);
        if (lane == 0) a.fit[d.fit_off + i] = fn;
    }
}

// Listed ties, one per CTA.  x - o and u - x are staged in shared memory,
// then every thread owns four rows of z = R (x - o) and dz = R (u - x) at
// once (four independent coalesced loads of R^T per column feed eight fma
// chains, so the L2 latency of streaming R^T is overlapped), and one warp
// forms the difference f(u) - f(x) (same difference forms as every other
// path).  With FP64 tie re-evaluation the rows are R (x - o) and R (u - o) in
// FP64 and the warp compares the two FP64 objectives.  Shared memory: 4 ws
// floats, or 4 ws doubles for FP64.
template <typename T>
__device__ __forceinline__ void tc_tie_rows(int dim, int dpad, const float* __restrict__ RT, const T* va,
                                            const T* vb, T* za, T* zb) {
    const int nt = blockDim.x;
    for (int r0 = threadIdx.x; r0 < dim; r0 += 4 * nt) {
        T aa[4] = {T(0), T(0), T(0), T(0)}, ab[4] = {T(0), T(0), T(0), T(0)};
        bool in[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) in[q] = r0 + q * nt < dim;
        for (int c = 0; c < dim; ++c) {
            const float* col = RT + (size_t)c * dpad + r0;
            const T xa = va[c], xb = vb[c];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (in[q]) {
                    const T rt = T(col[q * nt]);
                    aa[q] = fma(rt, xa, aa[q]);
                    ab[q] = fma(rt, xb, ab[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (in[q]) {
                za[r0 + q * nt] = aa[q];
                zb[r0 + q * nt] = ab[q];
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_tc_ties(StepArgs a, const int* __restrict__ row_exec,
                                                 const float* __restrict__ uscr, const int* __restrict__ tie_list,
                                                 const int* __restrict__ tie_count, int ws,
                                                 unsigned long long* tie_total) {
    extern __shared__ __align__(16) float smz[];
    __shared__ int take_s;
    __shared__ float fn_s;
    const int n = *tie_count;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(tie_total, (unsigned long long)n);
    for (int t = blockIdx.x; t < n; t += gridDim.x) {
        const int r = tie_list[t];
        const int k = row_exec[r];
        const InstDesc d = a.desc[k];
        const int i = r - d.tc_row;
        float* X = a.pop + d.pop_off + (long long)i * d.dpad;
        const float* U = uscr + d.pop_off + (long long)i * d.dpad;
        const float* o = a.shift + d.shift_off;
        const float* RT = a.rotT + d.rot_off;
        if (a.tie_fp64) {
            double* vx = reinterpret_cast<double*>(smz);
            double* vu = vx + ws;
            double* zx = vu + ws;
            double* zu = zx + ws;
            for (int c = threadIdx.x; c < d.dim; c += blockDim.x) {
                vx[c] = (double)X[c] - (double)o[c];
                vu[c] = (double)U[c] - (double)o[c];
            }
            __syncthreads();
            tc_tie_rows<double>(d.dim, d.dpad, RT, vx, vu, zx, zu);
            __syncthreads();
            if (threadIdx.x < 32) {
                const double eu = nan_to_inf(warp_objective<double>(d.obj, d.dim, zu));
                const double ex = nan_to_inf(warp_objective<double>(d.obj, d.dim, zx));
                if (threadIdx.x == 0) {
                    const float fx = a.fit[d.fit_off + i];
                    take_s = eu <= ex ? 1 : 0;
                    fn_s = fminf((float)eu, fx);
                }
            }
        } else {
            float* vx = smz;
            float* vl = vx + ws;
            float* zx = vl + ws;
            float* dz = zx + ws;
            for (int c = threadIdx.x; c < d.dim; c += blockDim.x) {
                const float xc = X[c];
                vx[c] = xc - o[c];
                vl[c] = U[c] - xc;
            }
            __syncthreads();
            tc_tie_rows<float>(d.dim, d.dpad, RT, vx, vl, zx, dz);
            __syncthreads();
            if (threadIdx.x < 32) {
                const float df = warp_diff(d.obj, d.dim, zx, dz);
                if (threadIdx.x == 0) {
                    const float fx = a.fit[d.fit_off + i];
                    take_s = df <= 0.0f ? 1 : 0;
                    fn_s = fx + df;
                }
            }
        }
        __syncthreads();
        if (take_s) {
            for (int j = threadIdx.x * 4; j < d.dpad; j += blockDim.x * 4)
                *reinterpret_cast<float4*>(X + j) = *reinterpret_cast<const float4*>(U + j);
            if (threadIdx.x == 0) a.fit[d.fit_off + i] = fn_s;
        }
        __syncthreads();
    }
}

// A operand rows of the population itself, x - o, for evaluating it on the
// tensor cores (initialisation).  Warp per row: x - o is staged in the warp's
// shared scratch (ws floats) and packed like a trial row.
__global__ void __launch_bounds__(256) k_tc_pack_pop(const InstDesc* __restrict__ desc,
                                                     const int* __restrict__ row_exec, int n_rows,
                                                     const float* __restrict__ pop, const float* __restrict__ shift,
                                                     int kp, void* aq, void* aq_lo, int ws, int fp8, float* ascale) {
    extern __shared__ __align__(16) float smp[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + warp;
    if (r >= n_rows) return;
    const InstDesc d = desc[row_exec[r]];
    const float* x = pop + d.pop_off + (long long)(r - d.tc_row) * d.dpad;
    const float* o = shift + d.shift_off;
    float* v = smp + (size_t)warp * ws;
    for (int j = lane; j < d.dim; j += 32) v[j] = x[j] - o[j];
    __syncwarp();
    pack_operand_row(v, d.dim, kp, aq, aq_lo, r, fp8, ascale + r);
}

// FP8: max |R| of one problem into *amax (as float bits; non-negative floats
// order like their bit patterns).  *amax must start at 0.
__global__ void k_tc_rot_amax(const float* __restrict__ rot, long long rot_off, int dim, int dpad, unsigned* amax) {
    float m = 0.0f;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)dim * dim;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / dim), c = (int)(e - (long long)r * dim);
        m = fmaxf(m, fabsf(rot[rot_off + (long long)r * dpad + c]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));
}

// B operand: padded R rows (rows >= dim and columns >= dim are zero).  BF16:
// hi, and the lo residual when split.  FP8: e4m3(R * 448 / max|R|), with the
// problem's max|R| / 448 written to *bscale by block 0.
__global__ void k_tc_pack_rot(const float* __restrict__ rot, long long rot_off, int dim, int dpad, int kp, void* bq,
                              void* bq_lo, long long brow, int fp8, const unsigned* amax, float* bscale) {
    const int r = blockIdx.x;
    if (fp8) {
        const float m = __uint_as_float(*amax);
        const float sc = m > 0.0f ? kE4M3Max / m : 1.0f;
        if (r == 0 && threadIdx.x == 0) *bscale = m > 0.0f ? m / kE4M3Max : 1.0f;
        uint8_t* row = reinterpret_cast<uint8_t*>(bq) + (brow + r) * kp;
        for (int c = threadIdx.x; c < kp; c += blockDim.x) {
            const float x = (r < dim && c < dim) ? rot[rot_off + (long long)r * dpad + c] : 0.0f;
            row[c] = (uint8_t)__nv_cvt_float_to_fp8(x * sc, __NV_SATFINITE, __NV_E4M3);
        }
        return;
    }
    __nv_bfloat16* row = reinterpret_cast<__nv_bfloat16*>(bq) + (brow + r) * kp;
    __nv_bfloat16* row_lo = bq_lo ? reinterpret_cast<__nv_bfloat16*>(bq_lo) + (brow + r) * kp : nullptr;
    for (int c = threadIdx.x; c < kp; c += blockDim.x) {
        const float x = (r < dim && c < dim) ? rot[rot_off + (long long)r * dpad + c] : 0.0f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        row[c] = hi;
        if (row_lo) row_lo[c] = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

// 2-D tensor map over a row-major [rows][kp] operand matrix of BF16 (esz 2)
// or e4m3 bytes (esz 1), box [128 bytes x box_rows], 128-byte swizzle,
// out-of-range rows read as zero.
bool tc_make_map(CUtensorMap* map, const void* base, long long rows, int kp, int box_rows, int esz) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * (cuuint64_t)esz};
    const cuuint32_t box[2] = {(cuuint32_t)(esz == 1 ? kBK8 : kBK), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, esz == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
              const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t tc_gemm_smem(bool split) { return (size_t)(split ? 2 : kStages) * (split ? 2 : 1) * (kAT + kBT) + 1024; }

cudaError_t launch_tc_pack_rot(const float* rot, long long rot_off, int dim, int dpad, int kp, int np_rows, void* bq,
                               void* bq_lo, long long brow, int fp8, unsigned* amax, float* bscale, cudaStream_t st) {
    if (fp8) {
        cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        k_tc_rot_amax<<<64, 256, 0, st>>>(rot, rot_off, dim, dpad, amax);
    }
    k_tc_pack_rot<<<np_rows, 256, 0, st>>>(rot, rot_off, dim, dpad, kp, bq, bq_lo, brow, fp8, amax, bscale);
    return cudaGetLastError();
}

cudaError_t launch_tc_eval(const InstDesc* desc, const TcPlan& p, const float* pop, const float* shift,
                           const float* rotT, float* fit, int* status, cudaStream_t st) {
    if (p.n_rows <= 0) return cudaSuccess;
    if (p.simt) return launch_rot_simt(desc, p.tiles, p.n_tiles, pop, shift, rotT, fit, p.max_dpad, st);
    const size_t smem_p = (size_t)8 * p.max_dpad * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_tc_pack_pop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p);
    if (e != cudaSuccess) return e;
    k_tc_pack_pop<<<(p.n_rows + 7) / 8, 256, smem_p, st>>>(desc, p.row_exec, p.n_rows, pop, shift, p.kp, p.aq,
                                                            p.split ? p.aq_lo : nullptr, p.max_dpad, p.fp8, p.ascale);
    const size_t smem_g = tc_gemm_smem(p.split);
    e = cudaFuncSetAttribute(k_rot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_g);
    if (e != cudaSuccess) return e;
    TcGemmArgs g;
    g.desc = desc;
    g.tiles = p.tiles;
    g.row_exec = p.row_exec;
    g.brow = p.brow;
    g.fu = fit;  // the epilogue writes f of each row straight into the fitness array
    g.kt = p.kp / (p.fp8 ? kBK8 : kBK);
    g.split = p.split;
    g.fp8 = p.fp8;
    g.ascale = p.ascale;
    g.bscale = p.bscale;
    g.status = status;
    g.sel = 0;
    k_rot_tc<<<p.n_tiles, kTcThreads, smem_g, st>>>(p.mapA, p.mapB, p.split ? p.mapAlo : p.mapA, p.split ? p.mapBlo : p.mapB,
                                             g);
    return cudaGetLastError();
}

cudaError_t launch_tc_trial_rows(const StepArgs& a, const TcPlan& p, cudaStream_t st) {
    k_tc_trial<<<(p.n_rows + 7) / 8, 256, 0, st>>>(a, p.row_exec, p.n_rows, p.topk_all, p.uscr, p.aq, nullptr,
                                                   p.kp, p.max_dpad, 0, p.ascale);
    return cudaGetLastError();
}

cudaError_t launch_rot_tc_select(const StepArgs& a, const TcPlan& p, cudaStream_t st) {
    const size_t smem_g = tc_gemm_smem(false);
    cudaError_t e = cudaFuncSetAttribute(k_rot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_g);
    if (e != cudaSuccess) return e;
    TcGemmArgs g;
    g.desc = a.desc;
    g.tiles = p.tiles;
    g.row_exec = p.row_exec;
    g.brow = p.brow;
    g.fu = p.fu;
    g.kt = p.kp / kBK;
    g.split = 0;
    g.fp8 = 0;
    g.ascale = p.ascale;
    g.bscale = p.bscale;
    g.status = a.status;
    g.sel = 1;
    g.pop = a.pop;
    g.fit = a.fit;
    g.uscr = p.uscr;
    g.theta = a.theta;
    g.prob_tp = p.prob_tp;
    g.tp_row0 = p.tp_row0;
    g.tie_cnt = p.tie_cnt;
    g.tie_list = p.tie_list;
    g.tie_off = p.tie_off;
    k_rot_tc<<<p.n_tiles, kTcThreads, smem_g, st>>>(p.mapA, p.mapB, p.mapA, p.mapB, g);
    return cudaGetLastError();
}

cudaError_t launch_wait_check(uint32_t rounds, int arrive, long long* out, int* status, cudaStream_t st) {
    k_wait_check<<<1, 32, 0, st>>>(rounds ? rounds : kWaitLimit, arrive, out, status);
    return cudaGetLastError();
}

cudaError_t launch_tc_generation(const StepArgs& a, const TcPlan& p, cudaStream_t st, cudaEvent_t* ev) {
    const bool batched = !a.tie_fp64;  // FP32 difference-form ties: listed per problem, batched kernels
    // narrow FP32 rows: k_tc_rank draws every row's indices into its draw record for k_tc_trial2
    const bool rows32 = p.simt && p.max_dpad <= 256;
    int4* trec = batched && rows32 ? p.trial_rec : nullptr;
    if (ev) cudaEventRecord(ev[0], st);
    if (batched) {
        cudaError_t e0 = launch_tc_rank(a, p, trec, st);  // also zeroes the per-problem tie counts
        if (e0 != cudaSuccess) return e0;
    } else {
        k_tc_prologue<<<p.n_exec, 256, 0, st>>>(a, p.execs, p.topk_all);
    }
    if (ev) cudaEventRecord(ev[1], st);
    const int blocks = (p.n_rows + 7) / 8;
    const size_t smem_t = p.fp8 ? (size_t)8 * p.max_dpad * sizeof(float) : 0;  // FP8 stages u - o per warp
    const size_t smem_s = (size_t)4 * p.max_dpad * (a.tie_fp64 ? sizeof(double) : sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(k_tc_trial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t);
    if (e != cudaSuccess) return e;
    if (rows32) {  // narrow FP32 rows: 16 rows per CTA, a lane per (row, 4 coordinates)
        e = launch_tc_trial_rows32(a, p, nullptr, trec, st);
        if (e != cudaSuccess) return e;
    } else {
        k_tc_trial<<<blocks, 256, smem_t, st>>>(a, p.row_exec, p.n_rows, p.topk_all, p.uscr, p.aq,
                                                p.split ? p.aq_lo : nullptr, p.kp, p.max_dpad, p.fp8, p.ascale);
    }
    if (p.simt) {
        if (ev) cudaEventRecord(ev[2], st);
        e = launch_rot_simt(a.desc, p.tiles, p.n_tiles, p.uscr, a.shift, a.rotT, p.fu, p.max_dpad, st);
        if (e != cudaSuccess) return e;
    } else {
        const size_t smem_g = tc_gemm_smem(p.split);
        e = cudaFuncSetAttribute(k_rot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_g);
        if (e != cudaSuccess) return e;
        TcGemmArgs g;
        g.desc = a.desc;
        g.tiles = p.tiles;
        g.row_exec = p.row_exec;
        g.brow = p.brow;
        g.fu = p.fu;
        g.kt = p.kp / (p.fp8 ? kBK8 : kBK);
        g.split = p.split;
        g.fp8 = p.fp8;
        g.ascale = p.ascale;
        g.bscale = p.bscale;
        g.status = a.status;
        g.sel = 0;
        if (ev) cudaEventRecord(ev[2], st);
        k_rot_tc<<<p.n_tiles, kTcThreads, smem_g, st>>>(p.mapA, p.mapB, p.split ? p.mapAlo : p.mapA, p.split ? p.mapBlo : p.mapB,
                                                 g);
    }
    if (ev) cudaEventRecord(ev[3], st);
    TieLists tl{};
    if (batched) {
        tl.prob_tp = p.prob_tp;
        tl.tp_row0 = p.tp_row0;
        tl.tie_cnt = p.tie_cnt;
        tl.tie_off = p.tie_off;
    } else {
        e = cudaMemsetAsync(p.tie_count, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
    }
    k_tc_select<<<blocks, 256, 0, st>>>(a, p.row_exec, p.n_rows, p.uscr, p.fu, p.tie_list, p.tie_count, tl);
    if (ev) cudaEventRecord(ev[4], st);
    if (batched) {
        e = launch_tc_ties_batched(a, p, st);
        if (e != cudaSuccess) return e;
    } else {
        e = cudaFuncSetAttribute(k_tc_ties, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s);
        if (e != cudaSuccess) return e;
        k_tc_ties<<<p.tie_ctas, 256, smem_s, st>>>(a, p.row_exec, p.uscr, p.tie_list, p.tie_count, p.max_dpad,
                                                   p.tie_total);
    }
    if (ev) cudaEventRecord(ev[5], st);
    return cudaGetLastError();
}

}  // namespace metade
