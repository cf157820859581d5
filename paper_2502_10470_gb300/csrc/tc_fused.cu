// tc_fused.cu -- one generation of the tensor-core executors in one kernel
// (BF16 operands, D <= 256), followed by a small commit kernel.
//
// k_tc_gen is persistent (one CTA per SM, 512 threads) and walks the 128-row
// M tiles of the GEMM (rows of one problem, possibly several executors).  Per
// tile:
//   1. draws      lanes 0..7 of every epilogue warp take one row each: the
//                 Philox index draws and K into a field-major record in shared
//                 memory; then each warp draws the exponential-crossover
//                 lengths of its 8 rows with all 32 lanes (a lane per four
//                 coordinate uniforms, the first one at or above CR found by a
//                 ballot);
//   2. trial      all 16 epilogue warps, a lane per (row, 4-coordinate chunk),
//                 8 rows x 4 consecutive chunks per warp step: mutation,
//                 crossover and clip (the same trial_chunk arithmetic as every
//                 other trial kernel), the FP32 trial row to global memory and
//                 the BF16 operand u - o straight into the A tile in shared
//                 memory, in the UMMA 128-byte-swizzled K-major layout (A never
//                 touches global memory);
//   3. MMA        thread 0 issues tcgen05.mma (M 128, N 256, K 16, FP32
//                 accumulate in TMEM) over the K tiles; B, the problem's padded
//                 BF16 R rows, is loaded by TMA once per problem and stays in
//                 shared memory while the CTA's tiles belong to that problem;
//   4. epilogue   16 warps read TMEM (tcgen05.ld), each a quarter of the
//                 columns of 32 rows, accumulate the objective and compose the
//                 quarters in column order (as the general GEMM does);
//   5. selection  a thread per row compares f(u) with the stored f(x); clear
//                 cases write the decision, near ties are listed;
//   6. ties       the tile's near ties, up to 16 at once: z = R (x - o) and
//                 dz = R (u - x) in FP32 on the CUDA cores (R^T streamed through
//                 shared memory by cp.async, once per batch), then the FP32
//                 difference form; a trial identical to its target is
//                 recognised from the staged u - x and accepted as it is.
// The decision goes to fu[fitness index]: the new fitness when the trial is
// accepted, NaN when it is rejected.  k_tc_commit (a CTA per executor) then
// copies the accepted rows, stores their fitness and ranks the pbest pool of
// the next generation; generational semantics hold because no row of the
// population changes before every trial of the generation is built.
//
// Every mbarrier wait is bounded; on timeout the kernel latches
// METADE_ETIMEOUT, waits (bounded) for its own TMA copy and MMAs, frees TMEM
// and returns.
#include "block.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace metade {

namespace {

using namespace tc;

constexpr int kRows = 128;       // rows per M tile (TMEM lanes)
constexpr int kMaxKt = 4;        // K tiles of 64 BF16 elements: D <= 256
constexpr int kTieBatch = 16;    // near ties rotated together
constexpr int kVec = 256;        // stride of a staged tie vector (floats)
constexpr int kRejected = -1;    // bit pattern of the "rejected" mark in fu (a NaN)
constexpr int kRtRows = 16;      // R^T rows per cp.async stage of the tie rotation
constexpr int kGenThreads = 32 * kEpiWarps;  // 16 warps; thread 0 also issues the TMA loads and MMAs

// record fields, [field][kRows]
enum {
    F_VALID, F_IBL, F_IBR, F_P0, F_P1, F_P2, F_P3, F_M0, F_M1, F_M2, F_M3, F_JR, F_NS, F_L, F_K,
    F_FIDX, F_POPLO, F_POPHI, F_F, F_CRI, F_PACK, F_I, F_STREAM, kFields
};

constexpr size_t kASize = (size_t)kMaxKt * kAT;                      // 64 KB
constexpr size_t kRecSize = (size_t)kFields * kRows * sizeof(int);   // 11.5 KB
constexpr size_t kPartSize = (size_t)(kParts - 1) * kRows * 8 * sizeof(float);  // 12 KB

struct GenArgs {
    StepArgs a;
    const int* tiles;         // [n_tiles][2]: first operand row, rows
    int n_tiles;
    const int* row_exec;      // operand row -> executor
    const long long* brow;    // per problem: first B row
    const int* topk_all;      // pbest pools (fitness layout)
    float* uscr;              // trial rows (population layout)
    float* fu;                // decisions (fitness layout)
    int kt;                   // K tiles of the operands
};

// 16-byte cp.async; src_bytes 0 fills the destination with zeros
__device__ __forceinline__ void cp_async16z(float* dst, const float* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// byte offset of 4 consecutive BF16 elements (k0, a multiple of 4) of row r in
// the 128-byte-swizzled K-major A tile: K tile k0 / 64, row r at r * 128,
// 16-byte unit (k0 % 64) / 8 at position unit ^ (r % 8), half (k0 % 8) / 4
__device__ __forceinline__ uint32_t a_off(int r, int k0) {
    return (uint32_t)((k0 >> 6) * kAT + r * 128 + ((((k0 & 63) >> 3) ^ (r & 7)) << 4) + ((k0 & 4) << 1));
}

__device__ __forceinline__ uint2 pack_bf16x4(const float (&d)[4]) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(d[0], d[1]);
    const __nv_bfloat162 hi = __floats2bfloat162_rn(d[2], d[3]);
    return make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
}

__global__ void __launch_bounds__(kGenThreads, 1) k_tc_gen(const __grid_constant__ CUtensorMap tmB, GenArgs g) {
    extern __shared__ uint8_t smraw[];
    __shared__ __align__(8) uint64_t bfull, mma_done, drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_s, ntie_s;
    __shared__ int tie_row[kRows];
    __shared__ float tie_fx[kRows];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    uint8_t* As = sm;
    uint8_t* Bs = sm + kASize;
    int* rec = reinterpret_cast<int*>(Bs + (size_t)g.kt * kBT);
    float* part = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(rec) + kRecSize);
    float* tv = reinterpret_cast<float*>(As);  // tie vectors reuse the A tile once the MMAs are done
    const StepArgs& a = g.a;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = tid == 0;  // TMA loads and MMAs
    const uint32_t epoch = a.epoch_dev ? *a.epoch_dev : a.epoch;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bfull, 1);
        mbar_init(&mma_done, 1);
        mbar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tmem_base;

    int cur_prob = -1;
    uint32_t bphase = 0, mphase = 0;
    bool b_in_flight = false;  // thread 0: a B load not yet waited on
    for (int t = blockIdx.x; t < g.n_tiles; t += gridDim.x) {
        const int arow = g.tiles[2 * t], nr = g.tiles[2 * t + 1];
        const InstDesc d = a.desc[g.row_exec[arow]];  // dim, objective and problem of every row of the tile
        // B: the problem's R rows, once per problem (the previous tile's MMAs are complete)
        const bool load_b = d.prob != cur_prob;
        if (load_b && issuer) {
            mbar_expect_tx(&bfull, (uint32_t)(g.kt * kBT));
            const int brow0 = (int)g.brow[d.prob];
            for (int kk = 0; kk < g.kt; ++kk) tma_load_2d(Bs + (size_t)kk * kBT, &tmB, &bfull, kk * kBK, brow0);
            b_in_flight = true;
        }
        cur_prob = d.prob;

        // 1. draws: warp w takes rows 8 w .. 8 w + 7; lanes 0..7 run a row's
        // index draws, then the warp's 32 lanes draw the exponential lengths of
        // its rows together (lane l: the uniforms of coordinates 4 l .. 4 l + 3)
        {
            const int r = 8 * warp + (lane & 7);
            int cs2 = 0;  // this lane's row uses exponential crossover
            if (lane < 8) {
                int valid = 0;
                if (r < nr) {
                    const int k = g.row_exec[arow + r];
                    const InstDesc e = a.desc[k];
                    const int i = arow + r - e.tc_row;
                    const Strat s = load_strat(a.theta + 6 * k, e.np);
                    if (s.ok) {
                        valid = 1;
                        cs2 = s.cs == 2;
                        const int* topk = g.topk_all + e.fit_off;
                        const Ctr c = make_ctr(a.key, (uint32_t)e.stream, a.gen0, (uint32_t)i, epoch);
                        Indiv v;
                        indiv_setup(s, c, i, e.np, e.dim, e.kp, topk, topk[0], v);
                        rec[F_IBL * kRows + r] = v.ibl;
                        rec[F_IBR * kRows + r] = v.ibr;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            rec[(F_P0 + q) * kRows + r] = q < s.dn ? diff_plus(v, s.a, q) : 0;
                            rec[(F_M0 + q) * kRows + r] = q < s.dn ? diff_minus(v, s.a, q) : 0;
                        }
                        rec[F_JR * kRows + r] = v.jrand;
                        rec[F_NS * kRows + r] = v.nstart;
                        rec[F_L * kRows + r] = 0;
                        rec[F_K * kRows + r] = (int)v.kraw;
                        rec[F_FIDX * kRows + r] = e.fit_off + i;
                        rec[F_POPLO * kRows + r] = (int)(uint32_t)e.pop_off;
                        rec[F_POPHI * kRows + r] = (int)(e.pop_off >> 32);
                        rec[F_F * kRows + r] = __float_as_int(s.F);
                        rec[F_CRI * kRows + r] = (int)s.cri;
                        rec[F_PACK * kRows + r] = s.cs | (s.dn << 4) | ((s.bl != s.br ? 1 : 0) << 8);
                        rec[F_I * kRows + r] = i;
                        rec[F_STREAM * kRows + r] = e.stream;
                    }
                }
                rec[F_VALID * kRows + r] = valid;
            }
            // exponential length L = 1 + min(t*, D - 1), t* the first coordinate
            // uniform U_t (slot 4 + t / 4, word t % 4) not below CR
            const unsigned exp_rows = __ballot_sync(kFull, cs2 != 0) & 0xFFu;
            __syncwarp();
            for (int base = 0; exp_rows && (base == 0 || base < d.dim - 1); base += 128) {  // t = base + 4 lane + q
                uint4 w8[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {  // the Philox chains of the 8 rows interleave
                    w8[q] = make_uint4(0, 0, 0, 0);
                    if ((exp_rows >> q) & 1u) {
                        const int rq = 8 * warp + q;
                        const Ctr c = make_ctr(a.key, (uint32_t)rec[F_STREAM * kRows + rq], a.gen0,
                                               (uint32_t)rec[F_I * kRows + rq], epoch);
                        w8[q] = c.slot(4 + (uint32_t)((base >> 2) + lane));
                    }
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (!((exp_rows >> q) & 1u)) continue;  // warp-uniform
                    const int rq = 8 * warp + q;
                    if (base > 0 && rec[F_L * kRows + rq] != 0) continue;  // ended in an earlier round
                    const uint32_t cri = (uint32_t)rec[F_CRI * kRows + rq];
                    int first = 4;  // first failing word of this lane
#pragma unroll
                    for (int wq = 3; wq >= 0; --wq) {
                        const int t = base + 4 * lane + wq;
                        if (t <= d.dim - 2 && (word_of(w8[q], wq) >> 8) >= cri) first = wq;
                    }
                    const unsigned fails = __ballot_sync(kFull, first < 4);
                    int L = 0;
                    if (fails) {
                        const int fl = __ffs(fails) - 1;
                        const int fq = __shfl_sync(kFull, first, fl);
                        L = 1 + base + 4 * fl + fq;
                    } else if (base + 128 >= d.dim - 1) {
                        L = d.dim;  // every uniform below CR: the whole row
                    }
                    if (lane == 0) rec[F_L * kRows + rq] = L;
                    __syncwarp();
                }
            }
        }
        __syncthreads();

        // 2. trial rows and the A tile: lane = (row 8 * unit + lane / 4, chunk 4 * unit' + lane % 4)
        {
            const int nchb = g.kt * 4;  // blocks of 4 chunks (16 elements) along K
            const int units = (kRows / 8) * nchb;
#pragma unroll 2
            for (int u = warp; u < units; u += kEpiWarps) {
                const int r = 8 * (u / nchb) + (lane >> 2);
                const int j4 = 4 * (4 * (u % nchb) + (lane & 3));
                float dd[4] = {0.f, 0.f, 0.f, 0.f};
                if (rec[F_VALID * kRows + r] && j4 < d.dpad) {
                    const long long po = (long long)(((unsigned long long)(uint32_t)rec[F_POPHI * kRows + r] << 32) |
                                                     (uint32_t)rec[F_POPLO * kRows + r]);
                    const float* X = a.pop + po;
                    const long long ld = d.dpad;
                    const int pack = rec[F_PACK * kRows + r];
                    Strat s;
                    s.F = __int_as_float(rec[F_F * kRows + r]);
                    s.cri = (uint32_t)rec[F_CRI * kRows + r];
                    s.cs = pack & 15;
                    s.dn = (pack >> 4) & 15;
                    s.bl = 0;
                    s.br = (pack >> 8) & 1;  // trial_chunk reads bl != br as "has a directional term"
                    const int i = rec[F_I * kRows + r];
                    // the population is read-only during the kernel: non-coherent loads, which the
                    // compiler may issue ahead of the previous unit's stores
                    const float4 av = __ldg(reinterpret_cast<const float4*>(X + rec[F_IBL * kRows + r] * ld + j4));
                    const float4 bv = __ldg(reinterpret_cast<const float4*>(X + rec[F_IBR * kRows + r] * ld + j4));
                    const float4 xv = __ldg(reinterpret_cast<const float4*>(X + (long long)i * ld + j4));
                    float4 p[4], m[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (q < s.dn) {
                            p[q] = __ldg(reinterpret_cast<const float4*>(X + rec[(F_P0 + q) * kRows + r] * ld + j4));
                            m[q] = __ldg(reinterpret_cast<const float4*>(X + rec[(F_M0 + q) * kRows + r] * ld + j4));
                        }
                    }
                    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (q < s.dn) {
                            sum.x += p[q].x - m[q].x; sum.y += p[q].y - m[q].y;
                            sum.z += p[q].z - m[q].z; sum.w += p[q].w - m[q].w;
                        }
                    }
                    uint4 w = make_uint4(0, 0, 0, 0);
                    if (s.cs == 1) {
                        const Ctr c = make_ctr(a.key, (uint32_t)rec[F_STREAM * kRows + r], a.gen0, (uint32_t)i, epoch);
                        w = c.slot(4 + (uint32_t)(j4 >> 2));
                    }
                    const float K = (float)(uint32_t)rec[F_K * kRows + r] * (1.0f / 16777216.0f);
                    float uo[4];
                    trial_chunk(s, K, rec[F_JR * kRows + r], rec[F_NS * kRows + r], rec[F_L * kRows + r], d.dim, j4,
                                av, bv, xv, sum, w, a.shift + d.shift_off, a.lo, a.hi, uo, dd);
                    *reinterpret_cast<float4*>(g.uscr + po + (long long)i * ld + j4) =
                        make_float4(uo[0], uo[1], uo[2], uo[3]);
                }
                *reinterpret_cast<uint2*>(As + a_off(r, j4)) = pack_bf16x4(dd);
            }
            fence_proxy_async();  // the generic-proxy writes of A become visible to the tensor cores
        }
        __syncthreads();

        // 3. MMA: one thread, over the K tiles, into one accumulator of kBN columns
        if (issuer) {
            bool ok = true;
            if (b_in_flight) {
                ok = mbar_wait(&bfull, bphase);
                bphase ^= 1u;
                b_in_flight = false;
            }
            if (ok) {
                tc_fence_after();
                for (int kk = 0; kk < g.kt; ++kk) {
                    const uint64_t ad = sdesc_sw128(smem_u32(As + (size_t)kk * kAT));
                    const uint64_t bd = sdesc_sw128(smem_u32(Bs + (size_t)kk * kBT));
#pragma unroll
                    for (int j = 0; j < kBK / 16; ++j)
                        mma_bf16(taddr, ad + 2 * j, bd + 2 * j, (kk > 0 || j > 0) ? 1u : 0u);
                }
                mma_commit(&mma_done);
            } else {
                set_status(a.status, kStatusTimeout);
                abort_s = 1;
            }
        }

        // 4. epilogue: warp w reads TMEM lanes 32 (w % 4).. and column part w / 4
        const int qd = warp & 3, prt = warp >> 2;
        const int row = 32 * qd + lane;
        ObjR acc;
        {
            const bool got = __all_sync(kFull, mbar_wait(&mma_done, mphase) ? 1 : 0) != 0;
            if (!got && lane == 0) {
                set_status(a.status, kStatusTimeout);
                abort_s = 1;
            }
            tc_fence_after();
            constexpr int kBpp = kBN / 32 / kParts;  // 32-column blocks per part
            float zf = 0.f, q1 = 0.f, qrun = 0.f;
            int nb = 0;
            if (got) {
                for (int pb = kBpp * prt; pb < kBpp * (prt + 1); ++pb) {
                    const int col0 = 32 * pb;
                    if (col0 >= d.dim) break;  // uniform across the warp
                    float v[32];
                    tmem_ld32(taddr + ((uint32_t)(32 * qd) << 16) + (uint32_t)col0, v);
                    if (prt) {
                        if (nb == 0) zf = v[0];
                        const int mcols = min(32, d.dim - col0);
                        if (d.obj == kSchwefel12) {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (j < mcols) {
                                    qrun += v[j];
                                    q1 += qrun;
                                }
                        }
                        nb += mcols;
                    }
                    acc.push32(d.obj, v, col0, d.dim);
                }
            }
            tc_fence_before();
            if (prt) {
                float* sl = part + ((size_t)(prt - 1) * kRows + row) * 8;
                *reinterpret_cast<float4*>(sl) = make_float4(acc.s0, acc.s1, acc.prev, acc.pre);
                *reinterpret_cast<float4*>(sl + 4) = make_float4(zf, q1, __int_as_float(nb), 0.f);
            }
        }
        mphase ^= 1u;
        __syncthreads();

        // 5. selection: the part-0 thread of each row
        if (tid == 0) ntie_s = 0;
        float fnew = 0.f;
        if (prt == 0) {
            for (int j = 0; j < kParts - 1; ++j) {
                const float* sl = part + ((size_t)j * kRows + row) * 8;
                const float4 x0 = *reinterpret_cast<const float4*>(sl), x1 = *reinterpret_cast<const float4*>(sl + 4);
                ObjR rb;
                rb.s0 = x0.x;
                rb.s1 = x0.y;
                rb.prev = x0.z;
                rb.pre = x0.w;
                rb.first = __float_as_int(x1.z) == 0;
                obj_compose(d.obj, acc, rb, x1.x, x1.y, __float_as_int(x1.z));
            }
            fnew = nan_to_inf(acc.finish(d.obj, d.dim));
        }
        __syncthreads();  // ntie_s = 0 before any tie is listed
        if (prt == 0 && rec[F_VALID * kRows + row] && !abort_s) {
            const int fidx = rec[F_FIDX * kRows + row];
            const float fx = a.fit[fidx];
            const float fn = fnew;
            // near ties (including trials identical to their targets, recognised
            // in the tie phase from the staged u - x) are decided below
            if (near_tie(fn, fx, tie_band(d.dim))) {
                const int q = atomicAdd(&ntie_s, 1);
                tie_row[q] = row;
                tie_fx[q] = fx;
            } else {
                g.fu[fidx] = fn <= fx ? fn : __int_as_float(kRejected);
            }
        }
        __syncthreads();

        // 6. near ties, kTieBatch at a time: z = R (x - o) and dz = R (u - x) in
        // FP32 (k ascending in every fma chain, like every FP32 rotation), R^T
        // streamed through shared memory 16 rows at a time by cp.async (double
        // buffered), each thread one row of z for half of the batch
        const int nt = abort_s ? 0 : ntie_s;
        const float* o = a.shift + d.shift_off;
        const float* RT = a.rotT + d.rot_off;
        float* vx = tv;                          // [kTieBatch][kVec] x - o, then z
        float* vl = tv + kTieBatch * kVec;       // u - x, then dz
        float* sR = tv + 2 * kTieBatch * kVec;   // [2][kRtRows][kVec] R^T rows
        const int nchunk = (d.dim + kRtRows - 1) / kRtRows;
        for (int b0 = 0; b0 < nt; b0 += kTieBatch) {
            const int nb = min(kTieBatch, nt - b0);
            auto stage_rt = [&](int ch) {  // R^T rows ch * 16 .. into buffer ch & 1 (zero past dim)
                float* dst = sR + (size_t)(ch & 1) * kRtRows * kVec;
                const int f4 = d.dpad >> 2;
                for (int e = tid; e < kRtRows * f4; e += blockDim.x) {
                    const int cc = e / f4, x4 = e - cc * f4, c = ch * kRtRows + cc;
                    cp_async16z(dst + cc * kVec + 4 * x4, RT + (size_t)min(c, d.dim - 1) * d.dpad + 4 * x4,
                                c < d.dim ? 16 : 0);
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            };
            stage_rt(0);
            for (int e = tid; e < nb * kVec; e += blockDim.x) {
                const int q = e / kVec, c = e - q * kVec;
                if (c < d.dpad) {
                    const int r = tie_row[b0 + q];
                    const long long po = (long long)(((unsigned long long)(uint32_t)rec[F_POPHI * kRows + r] << 32) |
                                                     (uint32_t)rec[F_POPLO * kRows + r]);
                    const long long off = po + (long long)rec[F_I * kRows + r] * d.dpad;
                    const float xc = a.pop[off + c];
                    vx[q * kVec + c] = c < d.dim ? xc - o[c] : 0.f;
                    vl[q * kVec + c] = g.uscr[off + c] - xc;
                }
            }
            const int r = tid & (kVec - 1), h = tid >> 8;  // row of z, half of the batch (h < 2)
            const int q0 = h * (kTieBatch / 2);
            float az[kTieBatch / 2], ad[kTieBatch / 2];
#pragma unroll
            for (int q = 0; q < kTieBatch / 2; ++q) az[q] = ad[q] = 0.f;
            for (int ch = 0; ch < nchunk; ++ch) {
                if (ch + 1 < nchunk) {
                    stage_rt(ch + 1);
                    asm volatile("cp.async.wait_group 1;" ::: "memory");
                } else {
                    asm volatile("cp.async.wait_group 0;" ::: "memory");
                }
                __syncthreads();
                if (h < 2 && r < d.dim) {
                    const float* rc = sR + (size_t)(ch & 1) * kRtRows * kVec;
                    const int cend = min(kRtRows, d.dim - ch * kRtRows);
                    for (int cc = 0; cc < cend; ++cc) {
                        const int c = ch * kRtRows + cc;
                        const float rt = rc[cc * kVec + r];
#pragma unroll
                        for (int q = 0; q < kTieBatch / 2; ++q) {
                            if (q0 + q < nb) {
                                az[q] = fmaf(rt, vx[(q0 + q) * kVec + c], az[q]);
                                ad[q] = fmaf(rt, vl[(q0 + q) * kVec + c], ad[q]);
                            }
                        }
                    }
                }
                __syncthreads();  // the buffer is refilled two chunks later
            }
            if (h < 2 && r < d.dim) {  // every thread has read vx / vl: z and dz replace them
#pragma unroll
                for (int q = 0; q < kTieBatch / 2; ++q) {
                    if (q0 + q < nb) {
                        vx[(q0 + q) * kVec + r] = az[q];
                        vl[(q0 + q) * kVec + r] = ad[q];
                    }
                }
            }
            __syncthreads();
            if (warp < nb) {
                // a trial identical to its target (u - x == 0 everywhere, pad included) is
                // accepted without evaluation; otherwise the FP32 difference form decides
                const int rr = tie_row[b0 + warp];
                const long long po = (long long)(((unsigned long long)(uint32_t)rec[F_POPHI * kRows + rr] << 32) |
                                                 (uint32_t)rec[F_POPLO * kRows + rr]);
                const long long off = po + (long long)rec[F_I * kRows + rr] * d.dpad;
                bool diff = false;
                for (int c = lane; c < d.dpad; c += 32) diff = diff || (g.uscr[off + c] != a.pop[off + c]);
                const float fx = tie_fx[b0 + warp];
                float dec;
                if (!__any_sync(kFull, diff)) {
                    dec = fx;
                } else {
                    const float df = warp_diff(d.obj, d.dim, vx + warp * kVec, vl + warp * kVec);
                    dec = df <= 0.0f ? fx + df : __int_as_float(kRejected);
                }
                if (lane == 0) g.fu[rec[F_FIDX * kRows + rr]] = dec;
            }
            __syncthreads();
        }
        if (abort_s) break;  // uniform: read after a barrier
        // the next tile's MMAs overwrite TMEM and A only after this barrier
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    // leave with no copy or MMA of this CTA in flight (bounded waits)
    if (issuer) {
        if (b_in_flight) mbar_wait(&bfull, bphase);
        mma_commit(&drain);
        mbar_wait(&drain, 0u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kBN) : "memory");
}

// Accepted rows into the population, their fitness, then the pbest pool of
// the next generation (block per executor; a warp per row for the copy).
__global__ void __launch_bounds__(256) k_tc_commit(StepArgs a, const int* __restrict__ execs, int* topk_all,
                                                   const float* __restrict__ uscr, const float* __restrict__ fu,
                                                   int rank_next) {
    const int k = execs[blockIdx.x];
    const InstDesc d = a.desc[k];
    const Strat s = load_strat(a.theta + 6 * k, d.np);
    if (!s.ok) {
        if (threadIdx.x == 0) set_status(a.status, 1);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < d.np; i += blockDim.x >> 5) {
        const float f = fu[d.fit_off + i];
        if (isnan(f)) continue;  // rejected (warp-uniform)
        float* X = a.pop + d.pop_off + (long long)i * d.dpad;
        const float* U = uscr + d.pop_off + (long long)i * d.dpad;
        for (int j = lane * 4; j < d.dpad; j += 128)
            *reinterpret_cast<float4*>(X + j) = *reinterpret_cast<const float4*>(U + j);
        if (lane == 0) a.fit[d.fit_off + i] = f;
    }
    if (!rank_next) return;
    __syncthreads();
    block_topk(a.fit + d.fit_off, d.np, d.kp, topk_all + d.fit_off);
}

__global__ void k_tc_rank(StepArgs a, const int* __restrict__ execs, int* topk_all) {
    const int k = execs[blockIdx.x];
    const InstDesc d = a.desc[k];
    const Strat s = load_strat(a.theta + 6 * k, d.np);
    if (!s.ok) {
        if (threadIdx.x == 0) set_status(a.status, 1);
        return;
    }
    block_topk(a.fit + d.fit_off, d.np, d.kp, topk_all + d.fit_off);
}

size_t gen_smem(int kt) { return 1024 + kASize + (size_t)kt * kBT + kRecSize + kPartSize; }

}  // namespace

bool tc_fused_fits(int kp) { return kp <= kMaxKt * kBK && gen_smem(kp / kBK) <= 227 * 1024; }

cudaError_t launch_tc_fused_generation(const StepArgs& a, const TcPlan& p, bool first, bool last, cudaStream_t st,
                                       cudaEvent_t* ev) {
    if (ev) cudaEventRecord(ev[0], st);
    if (first) k_tc_rank<<<p.n_exec, 256, 0, st>>>(a, p.execs, p.topk_all);
    if (ev) cudaEventRecord(ev[1], st);
    GenArgs g;
    g.a = a;
    g.tiles = p.tiles;
    g.n_tiles = p.n_tiles;
    g.row_exec = p.row_exec;
    g.brow = p.brow;
    g.topk_all = p.topk_all;
    g.uscr = p.uscr;
    g.fu = p.fu;
    g.kt = p.kp / kBK;
    const size_t smem = gen_smem(g.kt);
    cudaError_t e = cudaFuncSetAttribute(k_tc_gen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = p.n_tiles < p.gen_ctas ? p.n_tiles : p.gen_ctas;
    k_tc_gen<<<grid, kGenThreads, smem, st>>>(p.mapB, g);
    if (ev) cudaEventRecord(ev[2], st);
    k_tc_commit<<<p.n_exec, 256, 0, st>>>(a, p.execs, p.topk_all, p.uscr, p.fu, last ? 0 : 1);
    if (ev) cudaEventRecord(ev[3], st);
    return cudaGetLastError();
}

}  // namespace metade
