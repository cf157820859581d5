// tc_fused.cu -- one generation of the BF16 tensor-core executors (D <= 256)
// in four kernels, for the executors whose rotation is a small dense GEMM.
//
//   k_tc_rank   block per executor: best and the pbest pool from the stored
//               fitness (the generation-start ranking every trial uses), then
//               a thread per row: the row's Philox index draws, j_rand, the
//               exponential start and K, packed into a 64-byte draw record;
//   k_tc_trial2 a CTA of 128 threads per 16 operand rows, five resident per
//               SM.  Each warp reads the draw records of its four rows, then
//               draws their exponential-crossover lengths with its 32 lanes (a
//               lane per four coordinate uniforms, the first one at or above
//               CR found by a ballot); no barrier joins the warps.  (Without
//               records, as in the five-kernel pipeline, warp 0 runs the
//               index draws, a lane per row.)  Then a lane per (row,
//               4-coordinate chunk), 4 rows x 8 consecutive chunks per warp
//               step, the gathers of the next step in flight while this one is
//               built: mutation, crossover and clip (trial_chunk, the
//               arithmetic every trial kernel shares), the FP32 trial row and
//               the BF16 operand u - o, K-padded, to global memory.  The parent
//               offsets are re-read from shared memory at every step, which
//               leaves the registers to the loads in flight;
//   k_tc_sel    persistent, one CTA per SM, taking the 128-row M tiles
//               (rows of one problem, possibly of several executors) in
//               order from a counter, warp-specialised: a producer warp
//               reads the tile's entry of the tile table, issues the TMA
//               loads of the A tile and, where the problem changes, of B (the
//               problem's padded BF16 R rows, kept in shared memory while the
//               CTA's tiles belong to that problem) and the tcgen05.mma
//               (M 128, N 256, K 16, FP32 accumulate) into one of two TMEM
//               accumulators, so the loads and MMAs of tile j + 1 run during
//               the epilogue of tile j; 16 epilogue warps read TMEM
//               (tcgen05.ld), each a quarter of the columns of 32 rows,
//               accumulate the objective and compose the quarters in column
//               order; a thread per row then selects (its fitness index and
//               offsets from the row's draw record):
//               clear acceptances are committed at once (rows copied by the
//               whole CTA, four loads in flight per thread), near ties go to
//               their problem's tie list;
//   k_tc_ties2  the generation's near ties, 2 to 16 of one problem per chunk
//               (about one chunk per CTA), chunks spread over every SM by an
//               atomic counter: z = R (x -
//               o) and dz = R (u - x) in FP32 on the CUDA cores (R staged
//               through a 3-stage cp.async ring, float4 loads, every fma
//               chain in ascending k like every other FP32 rotation), the
//               FP32 difference form, and the commit; a trial identical to its
//               target is recognised from the staged u - x and accepted as it
//               is.  (Ties cluster: an executor whose F is near 0 has a tie in
//               almost every row, which one CTA per tile could not absorb.)
// Committing inside k_tc_sel and k_tc_ties2 keeps generational semantics:
// every trial row of the generation was built by k_tc_trial2 before they
// start, and each reads a population row only for that row's own decision.
// Results are bit-identical to the five-kernel pipeline of tc_rotate.cu.
//
// Every mbarrier wait is bounded; on timeout the kernel latches
// METADE_ETIMEOUT, waits (bounded) for its own TMA copies and MMAs, frees TMEM
// and returns.
#include "block.cuh"
#include "internal.h"
#include "tc_ptx.cuh"

namespace metade {

namespace {

using namespace tc;

constexpr int kRows = 128;                   // rows per M tile (TMEM lanes)
constexpr int kMaxKt = 4;                    // K tiles of 64 BF16 elements: D <= 256
constexpr int kSelThreads = 32 * kEpiWarps;  // 16 warps; thread 0 also issues the TMA loads and MMAs
constexpr int kTieBatch = 16;                // near ties rotated together
constexpr int kVec = 256;                    // stride of a staged tie vector (floats)
constexpr int kRc = 16;                      // R columns per cp.async stage of the tie rotation
constexpr int kRcs = kRc + 4;                // row stride of a stage: float4 loads of 8 rows hit 32 banks
constexpr int kRing = 3;                     // stages of the tie kernel's R ring (k_tc_ties2)
constexpr int kMaxTpSmem = 2048;             // problems whose chunk prefix k_tc_ties2 keeps in shared memory
constexpr int kTRows = 16;                   // rows per CTA of k_tc_trial2 (16 or 32)
constexpr int kTThreads = 8 * kTRows;        // a warp per four rows
constexpr int kTMinBlocks = 5;               // resident CTAs per SM the register budget is cut for

constexpr size_t kASize = (size_t)kMaxKt * kAT;                                  // 64 KB
constexpr size_t kPartSize = (size_t)(kParts - 1) * kRows * 8 * sizeof(float);  // 12 KB
constexpr size_t kTie2Size =
    (size_t)2 * kTieBatch * kVec * sizeof(float) + (size_t)kRing * kVec * kRcs * sizeof(float);  // 92 KB
static_assert((kASize + kPartSize) % 1024 == 0, "B must start 1024-byte aligned");

// record fields of k_tc_trial2, [field][kTRows]
enum {
    F_VALID, F_IBL, F_IBR, F_P0, F_P1, F_P2, F_P3, F_M0, F_M1, F_M2, F_M3, F_JR, F_NS, F_L, F_K,
    F_POPLO, F_POPHI, F_F, F_CRI, F_PACK, F_I, F_STREAM, F_DIM, F_DPAD, F_SHIFT, kFields
};

// 16-byte cp.async; src_bytes 0 fills the destination with zeros
__device__ __forceinline__ void cp_async16z(float* dst, const float* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ uint2 pack_bf16x4(const float (&d)[4]) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(d[0], d[1]);
    const __nv_bfloat162 hi = __floats2bfloat162_rn(d[2], d[3]);
    return make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
}

// ------------------------------------------------------------ k_tc_trial2
__global__ void __launch_bounds__(kTThreads, kTMinBlocks) k_tc_trial2(StepArgs a, const int* __restrict__ row_exec, int n_rows,
                                                         const int* __restrict__ topk_all, float* uscr, uint8_t* aq,
                                                         int kp, const int4* __restrict__ trec) {
    __shared__ int rec[kFields * kTRows];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.x * kTRows;
    const uint32_t epoch = a.epoch_dev ? *a.epoch_dev : a.epoch;

    // draws: from the rows' draw records (trec, written by k_tc_rank), warp w for its own rows
    // 4 w .. 4 w + 3, a lane per quarter record; or, without records, warp 0 with a lane per row.
    // Then the exponential lengths, warp w for rows 4 w .. 4 w + 3.
    if (trec) {
        const int r = 4 * warp + (lane >> 2), qp = lane & 3;
        if (lane < 16 && r0 + r < n_rows) {
            const int4 q = __ldg(trec + 4 * (size_t)(r0 + r) + qp);
            if (qp == 0) {
                rec[F_IBL * kTRows + r] = q.x & 0xFFFF;
                rec[F_IBR * kTRows + r] = q.x >> 16;
                rec[F_P0 * kTRows + r] = q.y & 0xFFFF;
                rec[F_M0 * kTRows + r] = q.y >> 16;
                rec[F_P1 * kTRows + r] = q.z & 0xFFFF;
                rec[F_M1 * kTRows + r] = q.z >> 16;
                rec[F_P2 * kTRows + r] = q.w & 0xFFFF;
                rec[F_M2 * kTRows + r] = q.w >> 16;
            } else if (qp == 1) {
                rec[F_P3 * kTRows + r] = q.x & 0xFFFF;
                rec[F_M3 * kTRows + r] = q.x >> 16;
                rec[F_JR * kTRows + r] = q.y & 0xFFFF;
                rec[F_NS * kTRows + r] = q.y >> 16;
                rec[F_K * kTRows + r] = q.z;
                rec[F_I * kTRows + r] = q.w & 0xFFFF;
                rec[F_PACK * kTRows + r] = (q.w >> 16) & 0xFFF;
                rec[F_VALID * kTRows + r] = (q.w >> 28) & 1;
                rec[F_L * kTRows + r] = 0;
            } else if (qp == 2) {
                rec[F_POPLO * kTRows + r] = q.x;
                rec[F_POPHI * kTRows + r] = q.y;
                rec[F_F * kTRows + r] = q.z;
                rec[F_CRI * kTRows + r] = q.w;
            } else {
                rec[F_STREAM * kTRows + r] = q.x;
                rec[F_DIM * kTRows + r] = q.y & 0xFFFF;
                rec[F_DPAD * kTRows + r] = q.y >> 16;
                rec[F_SHIFT * kTRows + r] = q.z;
            }
        } else if (lane < 16 && qp == 1) {
            rec[F_VALID * kTRows + r] = 0;  // past the last row: the exponential step skips it
        }
        __syncwarp();
    } else if (warp == 0 && lane < kTRows) {
        const int r = lane;
        {
            int valid = 0;
            if (r0 + r < n_rows) {
                const int k = row_exec[r0 + r];
                const InstDesc e = a.desc[k];
                const int i = r0 + r - e.tc_row;
                const Strat s = load_strat(a.theta + 6 * k, e.np);
                rec[F_DIM * kTRows + r] = e.dim;
                rec[F_DPAD * kTRows + r] = e.dpad;
                if (s.ok) {
                    valid = 1;
                    const int* topk = topk_all + e.fit_off;
                    const Ctr c = make_ctr(a.key, (uint32_t)e.stream, a.gen0, (uint32_t)i, epoch);
                    Indiv v;
                    indiv_setup(s, c, i, e.np, e.dim, e.kp, topk, topk[0], v);
                    rec[F_IBL * kTRows + r] = v.ibl;
                    rec[F_IBR * kTRows + r] = v.ibr;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        rec[(F_P0 + q) * kTRows + r] = q < s.dn ? diff_plus(v, s.a, q) : 0;
                        rec[(F_M0 + q) * kTRows + r] = q < s.dn ? diff_minus(v, s.a, q) : 0;
                    }
                    rec[F_JR * kTRows + r] = v.jrand;
                    rec[F_NS * kTRows + r] = v.nstart;
                    rec[F_L * kTRows + r] = 0;
                    rec[F_K * kTRows + r] = (int)v.kraw;
                    rec[F_POPLO * kTRows + r] = (int)(uint32_t)e.pop_off;
                    rec[F_POPHI * kTRows + r] = (int)(e.pop_off >> 32);
                    rec[F_F * kTRows + r] = __float_as_int(s.F);
                    rec[F_CRI * kTRows + r] = (int)s.cri;
                    rec[F_PACK * kTRows + r] = s.cs | (s.dn << 4) | ((s.bl != s.br ? 1 : 0) << 8);
                    rec[F_I * kTRows + r] = i;
                    rec[F_STREAM * kTRows + r] = e.stream;
                    rec[F_SHIFT * kTRows + r] = e.shift_off;
                }
            }
            rec[F_VALID * kTRows + r] = valid;
        }
    }
    if (trec) __syncwarp();  // uniform over the CTA: every warp reads only its own rows
    else __syncthreads();
    {
        // exponential length L = 1 + min(t*, D - 1), t* the first coordinate
        // uniform U_t (slot 4 + t / 4, word t % 4) not below CR
        const int r = 4 * warp + (lane & 3);
        const bool cs2 = lane < 4 && rec[F_VALID * kTRows + r] && (rec[F_PACK * kTRows + r] & 15) == 2;
        const unsigned exp_rows = __ballot_sync(kFull, cs2) & 0xFu;
        if (exp_rows) {
            int dmax = 0;  // the widest exponential row of the warp bounds the rounds
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if ((exp_rows >> q) & 1u) dmax = max(dmax, rec[F_DIM * kTRows + 4 * warp + q]);
            for (int base = 0; base == 0 || base < dmax - 1; base += 128) {  // t = base + 4 lane + word
                uint4 w4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {  // the Philox chains of the four rows interleave
                    w4[q] = make_uint4(0, 0, 0, 0);
                    if ((exp_rows >> q) & 1u) {
                        const int rq = 4 * warp + q;
                        const Ctr c = make_ctr(a.key, (uint32_t)rec[F_STREAM * kTRows + rq], a.gen0,
                                               (uint32_t)rec[F_I * kTRows + rq], epoch);
                        w4[q] = c.slot(4 + (uint32_t)((base >> 2) + lane));
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (!((exp_rows >> q) & 1u)) continue;  // warp-uniform
                    const int rq = 4 * warp + q;
                    const int dim = rec[F_DIM * kTRows + rq];
                    if (rec[F_L * kTRows + rq] != 0 || (base > 0 && base >= dim - 1)) continue;  // done
                    const uint32_t cri = (uint32_t)rec[F_CRI * kTRows + rq];
                    int first = 4;  // first failing word of this lane
#pragma unroll
                    for (int wq = 3; wq >= 0; --wq) {
                        const int t = base + 4 * lane + wq;
                        if (t <= dim - 2 && (word_of(w4[q], wq) >> 8) >= cri) first = wq;
                    }
                    const unsigned fails = __ballot_sync(kFull, first < 4);
                    int L = 0;
                    if (fails) {
                        const int fl = __ffs(fails) - 1;
                        const int fq = __shfl_sync(kFull, first, fl);
                        L = 1 + base + 4 * fl + fq;
                    } else if (base + 128 >= dim - 1) {
                        L = dim;  // every uniform below CR: the whole row
                    }
                    if (lane == 0) rec[F_L * kTRows + rq] = L;
                    __syncwarp();
                }
            }
        }
    }
    if (trec) __syncwarp();
    else __syncthreads();

    // trial rows and operand rows: warp w takes rows 4 w + lane / 8 and every
    // 32-element column block of them; lane % 8 picks the chunk of four elements,
    // so eight lanes read and write a whole 128-byte line of a row at a time.  A
    // lane keeps its row's fields in registers across its chunks.
    const int r = 4 * warp + (lane >> 3);
    if (r0 + r >= n_rows) return;  // no barrier follows
    uint8_t* arow = aq ? aq + (size_t)(r0 + r) * kp * 2 : nullptr;  // null: FP32 GEMM, no operand rows
    const int dpad = rec[F_DPAD * kTRows + r];
    // blocks of 8 chunks along K, up to the row's own K tiles (k_tc_sel reads no further)
    const int nchb = ((dpad + kBK - 1) / kBK) * (kBK / 32);
    if (!rec[F_VALID * kTRows + r]) {  // rows of an invalid theta: a zero operand row
        if (!arow) return;
        for (int cb = 0; cb < nchb; ++cb)
            *reinterpret_cast<uint2*>(arow + (size_t)(4 * (8 * cb + (lane & 7))) * 2) = make_uint2(0u, 0u);
        return;
    }
    const long long po = (long long)(((unsigned long long)(uint32_t)rec[F_POPHI * kTRows + r] << 32) |
                                     (uint32_t)rec[F_POPLO * kTRows + r]);
    const float* X = a.pop + po;
    const int pack = rec[F_PACK * kTRows + r];
    Strat s;
    s.F = __int_as_float(rec[F_F * kTRows + r]);
    s.cri = (uint32_t)rec[F_CRI * kTRows + r];
    s.cs = pack & 15;
    s.dn = (pack >> 4) & 15;
    s.bl = 0;
    s.br = (pack >> 8) & 1;  // trial_chunk reads bl != br as "has a directional term"
    const int i = rec[F_I * kTRows + r];
    // parent rows as float offsets from X (an executor holds at most 1024 x 1536 floats)
    const int oi = i * dpad;
    const int jr = rec[F_JR * kTRows + r], ns = rec[F_NS * kTRows + r], L = rec[F_L * kTRows + r];
    const int dim = rec[F_DIM * kTRows + r];
    const float* o = a.shift + rec[F_SHIFT * kTRows + r];
    const float K = (float)(uint32_t)rec[F_K * kTRows + r] * (1.0f / 16777216.0f);
    const Ctr c = make_ctr(a.key, (uint32_t)rec[F_STREAM * kTRows + r], a.gen0, (uint32_t)i, epoch);
    float* U = uscr + po + oi;
    // The gathers are software-pipelined along the row: the parent chunks of
    // block cb + 1 are loaded (the population is read-only here: non-coherent
    // loads) while block cb is built, so a lane keeps two blocks in flight.
    float4 ga, gb, gx, gp[4], gm[4];
    // The parent row indices are re-read from the shared record at every
    // block (volatile: not held in registers across the loop), which leaves
    // the registers to the loads in flight.
    const volatile int* vr = rec + r;
    auto issue = [&](int j4) {
        if (j4 < dpad) {
            ga = __ldg(reinterpret_cast<const float4*>(X + vr[F_IBL * kTRows] * dpad + j4));
            gb = __ldg(reinterpret_cast<const float4*>(X + vr[F_IBR * kTRows] * dpad + j4));
            gx = __ldg(reinterpret_cast<const float4*>(X + oi + j4));
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q < s.dn) {
                    gp[q] = __ldg(reinterpret_cast<const float4*>(X + vr[(F_P0 + q) * kTRows] * dpad + j4));
                    gm[q] = __ldg(reinterpret_cast<const float4*>(X + vr[(F_M0 + q) * kTRows] * dpad + j4));
                }
            }
        }
    };
    issue(4 * (lane & 7));
    for (int cb = 0; cb < nchb; ++cb) {
        const int j4 = 4 * (8 * cb + (lane & 7));
        float dd[4] = {0.f, 0.f, 0.f, 0.f};
        const float4 av = ga, bv = gb, xv = gx;
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j4 < dpad) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q < s.dn) {
                    sum.x += gp[q].x - gm[q].x; sum.y += gp[q].y - gm[q].y;
                    sum.z += gp[q].z - gm[q].z; sum.w += gp[q].w - gm[q].w;
                }
            }
        }
        if (cb + 1 < nchb) issue(j4 + 32);
        if (j4 < dpad) {
            const uint4 w = s.cs == 1 ? c.slot(4 + (uint32_t)(j4 >> 2)) : make_uint4(0, 0, 0, 0);
            float uo[4];
            trial_chunk(s, K, jr, ns, L, dim, j4, av, bv, xv, sum, w, o, a.lo, a.hi, uo, dd);
            *reinterpret_cast<float4*>(U + j4) = make_float4(uo[0], uo[1], uo[2], uo[3]);
        }
        if (arow) *reinterpret_cast<uint2*>(arow + (size_t)j4 * 2) = pack_bf16x4(dd);
    }
}

// --------------------------------------------------------------- k_tc_sel
// The accepted rows of a tile copied from the trial rows (src) into the population (dst) by nt
// threads, element e = (row e / f4, float4 e % f4): each thread issues eight loads before their
// stores, so the copy takes one memory round trip per eight of its elements rather than per one.
__device__ __forceinline__ void copy_accepted(const long long* offs, int nrows, int f4, const float* src, float* dst,
                                              int t, int nt) {
    const int n = nrows * f4;
    for (int e0 = t; e0 < n; e0 += 4 * nt) {
        float4 v[4];
        long long off[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e2 = e0 + u * nt;
            off[u] = 0;
            if (e2 < n) {
                const int q = e2 / f4, c4 = e2 - q * f4;
                off[u] = offs[q] + 4 * c4;
                v[u] = __ldg(reinterpret_cast<const float4*>(src + off[u]));
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (e0 + u * nt < n) *reinterpret_cast<float4*>(dst + off[u]) = v[u];
    }
}

struct SelArgs {
    StepArgs a;
    const int* tiles;         // [n_tiles][2]: first operand row, rows (all of one problem)
    int n_tiles;
    int* next_tile;           // tiles handed out beyond the first gridDim.x (zeroed by k_tc_rank)
    const int* prob_tp;       // problem -> index among the problems on this path
    const int* tp_row0;       // per such problem: its first operand row (start of its tie list)
    int* tie_cnt;             // per such problem: near ties listed (zeroed by k_tc_rank)
    int* tie_list;            // fitness index of each near tie, by problem
    long long* tie_off;       // population offset of each near tie's row, by problem
    const int* row_exec;      // operand row -> executor
    const long long* brow;    // per problem: first B row
    const float* uscr;        // trial rows (population layout)
    int kt;                   // K tiles of the widest problem (shared memory is cut for it)
    const int4* tmeta;        // [n_tiles][2]: (first row, rows, D, D_pad), (objective, problem, 0, 0)
    const int4* trec;         // the rows' draw records (k_tc_rank): validity, fitness index, offsets
};

// Named barrier of the 16 epilogue warps (the producer warp does not take part).
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kSelThreads) : "memory"); }

__global__ void __launch_bounds__(kSelThreads + 32, 1) k_tc_sel(const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB, SelArgs g) {
    extern __shared__ uint8_t smraw[];
    __shared__ __align__(8) uint64_t afull, bfull, acc_full[2], acc_empty[2], drain, tile_ready[2];
    __shared__ uint32_t tmem_base;
    __shared__ int ep_abort_s, nacc_s, tile_of[2];  // tile in accumulator b (-1: no more tiles)
    __shared__ int tinfo[2][6];  // that tile's first row, rows, D, D_pad, objective, problem (posted with it)
    __shared__ long long acc_off[kRows];  // population offsets of the tile's accepted rows
    __shared__ float gk[kBN];             // Griewank's factor 1 / (2 pi sqrt(j + 1)) of column j
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    uint8_t* As = sm;
    float* part = reinterpret_cast<float*>(sm + kASize);
    uint8_t* Bs = sm + kASize + kPartSize;
    const StepArgs& a = g.a;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * kBN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&afull, 1);
        mbar_init(&bfull, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kEpiWarps);  // one arrival per epilogue warp
            mbar_init(&tile_ready[b], 1);
        }
        mbar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        ep_abort_s = 0;
    }
    for (int j = tid; j < kBN; j += blockDim.x) gk[j] = rsqrtf((float)(j + 1)) * kInv2Pi;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tmem_base;
    // Tiles are handed out in order (blockIdx.x first, then an atomic counter): tiles differ in
    // cost (D, the objective, the accepted rows to copy), and consecutive tiles mostly belong to
    // one problem (its tiles are adjacent), so B is reloaded only where the problem changes.  The
    // producer posts each tile's index per accumulator (tile_ready), -1 when none is left.

    if (warp == kEpiWarps) {
        // producer: A of tile j (and B at a new problem) once the MMAs of tile j - 1 are done with
        // the shared memory, then the MMAs of tile j into accumulator j % 2 once the epilogue has
        // released it (tile j - 2), so they overlap the epilogue of tile j - 1
        if (lane == 0) {
            int cur_prob = -1;
            uint32_t aphase = 0, bphase = 0;
            bool ok = true, a_fly = false, b_fly = false, mma_any = false;
            int j = 0;
            bool posted = false;  // tile j's index is posted
            for (;; ++j) {
                const int b = j & 1;
                posted = false;
                // tile j, claimed when it is due (claiming one tile ahead measured slower), and its
                // entry of the tile table
                const int t = j == 0 ? (int)blockIdx.x : (int)gridDim.x + atomicAdd(g.next_tile, 1);
                int4 m0 = make_int4(0, 0, 0, 0), m1 = m0;
                if (t < g.n_tiles) {
                    m0 = __ldg(g.tmeta + 2 * t);
                    m1 = __ldg(g.tmeta + 2 * t + 1);
                }
                // accumulator b's slot is free once the epilogue released tile j - 2
                if (j >= 2 && !mbar_wait(&acc_empty[b], (uint32_t)((j - 2) >> 1) & 1u)) {
                    ok = false;
                    break;
                }
                posted = true;
                const int arow = m0.x;
                struct {
                    int dim, dpad, obj, prob;
                } d = {m0.z, m0.w, m1.x, m1.y};  // of every row of the tile
                if (t < g.n_tiles) {
                    tinfo[b][0] = arow;
                    tinfo[b][1] = m0.y;
                    tinfo[b][2] = d.dim;
                    tinfo[b][3] = d.dpad;
                    tinfo[b][4] = d.obj;
                    tinfo[b][5] = d.prob;
                }
                tile_of[b] = t < g.n_tiles ? t : -1;
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tile_ready[b])) : "memory");
                if (t >= g.n_tiles) break;
                const int kt = (d.dpad + kBK - 1) / kBK;
                if (j > 0 && !mbar_wait(&acc_full[(j - 1) & 1], (uint32_t)((j - 1) >> 1) & 1u)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(&afull, (uint32_t)(kt * kAT));
                for (int kk = 0; kk < kt; ++kk) tma_load_2d(As + (size_t)kk * kAT, &tmA, &afull, kk * kBK, arow);
                a_fly = true;
                if (d.prob != cur_prob) {
                    mbar_expect_tx(&bfull, (uint32_t)(kt * kBT));
                    const int brow0 = (int)g.brow[d.prob];
                    for (int kk = 0; kk < kt; ++kk)
                        tma_load_2d(Bs + (size_t)kk * kBT, &tmB, &bfull, kk * kBK, brow0);
                    b_fly = true;
                    cur_prob = d.prob;
                }
                ok = mbar_wait(&afull, aphase);
                aphase ^= 1u;
                a_fly = false;
                if (ok && b_fly) {
                    ok = mbar_wait(&bfull, bphase);
                    bphase ^= 1u;
                    b_fly = false;
                }
                if (!ok) break;
                tc_fence_after();
                const uint32_t dacc = taddr + (uint32_t)(b * kBN);
                for (int kk = 0; kk < kt; ++kk) {
                    const uint64_t ad = sdesc_sw128(smem_u32(As + (size_t)kk * kAT));
                    const uint64_t bd = sdesc_sw128(smem_u32(Bs + (size_t)kk * kBT));
#pragma unroll
                    for (int q = 0; q < kBK / 16; ++q) mma_bf16(dacc, ad + 2 * q, bd + 2 * q, (kk > 0 || q > 0) ? 1u : 0u);
                }
                mma_commit(&acc_full[b]);
                mma_any = true;
            }
            if (!ok) {
                set_status(a.status, kStatusTimeout);
                // a tile that was posted ends the epilogue by its own bounded wait on acc_full; an
                // unposted slot gets -1, so the epilogue stops there (it read the slot's old index
                // before releasing tile j - 2, or never got that far)
                if (!posted) {
                    tile_of[j & 1] = -1;
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tile_ready[j & 1]))
                                 : "memory");
                }
            }
            // leave with no copy or MMA of this CTA in flight (bounded waits)
            if (a_fly) mbar_wait(&afull, aphase);
            if (b_fly) mbar_wait(&bfull, bphase);
            if (mma_any) {
                mma_commit(&drain);
                mbar_wait(&drain, 0u);
            }
        }
        __syncwarp();
    } else {
        // epilogue warps: warp w reads TMEM lanes 32 (w % 4).. and column part w / 4
        const int qd = warp & 3, prt = warp >> 2;
        const int row = 32 * qd + lane;
        for (int j = 0;; ++j) {
            const int b = j & 1;
            if (!__all_sync(kFull, mbar_wait(&tile_ready[b], (uint32_t)(j >> 1) & 1u) ? 1 : 0)) {  // bounded
                if (lane == 0) set_status(a.status, kStatusTimeout);
                break;
            }
            const int t = tile_of[b];
            if (t < 0) break;  // the same for every epilogue warp
            const int arow = tinfo[b][0], nr = tinfo[b][1];
            struct {
                int dim, dpad, obj, prob;
            } d = {tinfo[b][2], tinfo[b][3], tinfo[b][4], tinfo[b][5]};  // of every row of the tile
            // the row's executor fields and stored fitness, fetched before the TMEM work so that these
            // dependent loads overlap it (part-0 threads, which select)
            bool rok = false;
            int fidx = 0;
            long long roff = 0;
            float fx = 0.f;
            if (prt == 0 && row < nr) {  // from the row's draw record: one level of loads
                const int4* rq = g.trec + 4 * (size_t)(arow + row);
                const int4 q1 = __ldg(rq + 1), q2 = __ldg(rq + 2), q3 = __ldg(rq + 3);
                rok = (q1.w >> 28) & 1;  // rows of an invalid theta stay as they are
                fidx = q3.w;
                roff = (long long)(((unsigned long long)(uint32_t)q2.y << 32) | (uint32_t)q2.x) +
                       (long long)(q1.w & 0xFFFF) * d.dpad;
                if (rok) fx = a.fit[fidx];
            }
            ObjR acc;
            const bool got = __all_sync(kFull, mbar_wait(&acc_full[b], (uint32_t)(j >> 1) & 1u) ? 1 : 0) != 0;
            tc_fence_after();
            constexpr int kBpp = kBN / 32 / kParts;  // 32-column blocks per part
            float zf = 0.f, q1 = 0.f, qrun = 0.f;
            int nb = 0;
            if (got) {
                for (int pb = kBpp * prt; pb < kBpp * (prt + 1); ++pb) {
                    const int col0 = 32 * pb;
                    if (col0 >= d.dim) break;  // uniform across the warp
                    float v[32];
                    tmem_ld32(taddr + ((uint32_t)(32 * qd) << 16) + (uint32_t)(b * kBN + col0), v);
                    if (prt) {
                        if (nb == 0) zf = v[0];
                        const int mcols = min(32, d.dim - col0);
                        if (d.obj == kSchwefel12) {
#pragma unroll
                            for (int q = 0; q < 32; ++q)
                                if (q < mcols) {
                                    qrun += v[q];
                                    q1 += qrun;
                                }
                        }
                        nb += mcols;
                    }
                    if (d.obj == kGriewank) acc.push32_griewank(v, col0, d.dim, gk + col0);
                    else acc.push32(d.obj, v, col0, d.dim);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {  // this warp has read the accumulator: the producer may reuse it
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
                if (!got) {
                    set_status(a.status, kStatusTimeout);
                    ep_abort_s = 1;
                }
            }
            if (prt) {
                float* sl = part + ((size_t)(prt - 1) * kRows + row) * 8;
                *reinterpret_cast<float4*>(sl) = make_float4(acc.s0, acc.s1, acc.prev, acc.pre);
                *reinterpret_cast<float4*>(sl + 4) = make_float4(zf, q1, __int_as_float(nb), 0.f);
            }
            if (tid == 0) nacc_s = 0;
            epi_sync();
            if (ep_abort_s) break;  // uniform: read after the barrier

            // selection: the part-0 thread of each row; clear acceptances are listed for the row
            // copy, near ties go to the problem's tie list (k_tc_ties2)
            if (prt == 0 && row < nr) {
                for (int q = 0; q < kParts - 1; ++q) {
                    const float* sl = part + ((size_t)q * kRows + row) * 8;
                    const float4 x0 = *reinterpret_cast<const float4*>(sl), x1 = *reinterpret_cast<const float4*>(sl + 4);
                    ObjR rb;
                    rb.s0 = x0.x;
                    rb.s1 = x0.y;
                    rb.prev = x0.z;
                    rb.pre = x0.w;
                    rb.first = __float_as_int(x1.z) == 0;
                    obj_compose(d.obj, acc, rb, x1.x, x1.y, __float_as_int(x1.z));
                }
                const float fn = nan_to_inf(acc.finish(d.obj, d.dim));
                if (rok) {
                    if (near_tie(fn, fx, tie_band(d.dim))) {
                        const int tp = g.prob_tp[d.prob];
                        const int q = g.tp_row0[tp] + atomicAdd(&g.tie_cnt[tp], 1);
                        g.tie_list[q] = fidx;
                        g.tie_off[q] = roff;
                    } else if (fn <= fx) {
                        acc_off[atomicAdd(&nacc_s, 1)] = roff;
                        a.fit[fidx] = fn;
                    }
                }
            }
            epi_sync();
            // accepted rows into the population, copied by the 16 warps
            copy_accepted(acc_off, nacc_s, d.dpad >> 2, g.uscr, a.pop, tid, kSelThreads);
            epi_sync();  // acc_off and the exchange area are reused by the next tile
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(2 * kBN) : "memory");
}

// -------------------------------------------------------------- k_tc_ties2
struct TieArgs {
    StepArgs a;
    const int* row_exec;      // operand row -> executor
    int n_tp;                 // problems on this path
    const int* tp_row0;       // per problem: its first operand row (start of its tie list)
    const int* tie_cnt;       // per problem: near ties listed by k_tc_sel
    const int* tie_list;      // fitness index of each near tie, by problem
    const long long* tie_off; // population offset of each near tie's row, by problem
    int* chunk_ctr;           // chunks handed out (zeroed by k_tc_rank)
    const float* uscr;        // trial rows (population layout)
    unsigned long long* tie_total;  // near ties decided, summed over generations (block 0 adds)
};

// The near ties of the generation, up to kTieBatch ties of one problem per
// chunk (fewer when ties are few), chunks handed out by an atomic counter
// over every CTA of the GPU (two per SM): z = R (x - o) and dz = R (u - x)
// in FP32, R staged through shared memory 16 columns at a time by cp.async
// in a ring of kRing stages, a thread per (two rows of z, group of the
// chunk's ties; the narrower the problem, the more groups) with float4 loads
// along k, every fma chain in ascending k; then a warp per tie forms the FP32
// difference form f(u) - f(x), decides and commits.  A trial identical to
// its target (u - x == 0 everywhere, pad included) is accepted as it is.
__global__ void __launch_bounds__(kSelThreads, 2) k_tc_ties2(TieArgs g) {
    extern __shared__ uint8_t smraw[];
    __shared__ int tp_s, j0_s, bsz_s, ncum_s[kMaxTpSmem + 1];
    float* tv = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 15) & ~(uintptr_t)15);
    const StepArgs& a = g.a;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float* vx = tv;                          // [kTieBatch][kVec] x - o, then z
    float* vl = tv + kTieBatch * kVec;       // u - x, then dz
    float* sR = tv + 2 * kTieBatch * kVec;   // [kRing][kVec][kRcs]: R columns c0 .. c0 + 15 of every row
    // chunk size: as few whole rounds of chunks over the grid as full chunks need, filled evenly
    // (few ties: small chunks, so no SM waits behind another's long chunk), between 2 and
    // kTieBatch; every CTA derives the same size from the same final counts (k_tc_sel has ended)
    if (tid == 0) {
        long long total = 0;
        for (int q = 0; q < g.n_tp; ++q) total += g.tie_cnt[q];
        // rounds of chunks over the grid at full chunks, then the chunk that fills those rounds evenly
        const long long rounds = max(1LL, (total + (long long)gridDim.x * kTieBatch - 1) / ((long long)gridDim.x * kTieBatch));
        const long long per = (long long)gridDim.x * rounds;
        bsz_s = (int)min((long long)kTieBatch, max(2LL, (total + per - 1) / per));
        if (blockIdx.x == 0) atomicAdd(g.tie_total, (unsigned long long)total);
    }
    __syncthreads();
    const int bsz = bsz_s;
    // chunks per problem, summed in problem order
    const bool cum_smem = g.n_tp <= kMaxTpSmem;
    if (cum_smem) {
        for (int q = tid; q < g.n_tp; q += blockDim.x) ncum_s[q + 1] = (g.tie_cnt[q] + bsz - 1) / bsz;
        __syncthreads();
        if (tid == 0) {
            ncum_s[0] = 0;
            for (int q = 0; q < g.n_tp; ++q) ncum_s[q + 1] += ncum_s[q];
        }
        __syncthreads();
    }
    for (;;) {
        if (tid == 0) {  // chunk c -> (problem, first tie)
            const int c = atomicAdd(g.chunk_ctr, 1);
            int tp = -1, j0 = 0;
            if (cum_smem) {
                if (c < ncum_s[g.n_tp]) {  // the last problem whose first chunk is <= c
                    int lo = 0, hi = g.n_tp - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (ncum_s[mid] <= c) lo = mid;
                        else hi = mid - 1;
                    }
                    tp = lo;
                    j0 = (c - ncum_s[lo]) * bsz;
                }
            } else {
                int acc = 0;
                for (int q = 0; q < g.n_tp; ++q) {
                    const int n = (g.tie_cnt[q] + bsz - 1) / bsz;
                    if (c < acc + n) {
                        tp = q;
                        j0 = (c - acc) * bsz;
                        break;
                    }
                    acc += n;
                }
            }
            tp_s = tp;
            j0_s = j0;
        }
        __syncthreads();
        const int tp = tp_s, j0 = j0_s;
        if (tp < 0) break;
        const int nb = min(bsz, g.tie_cnt[tp] - j0);
        const int* tfid = g.tie_list + g.tp_row0[tp] + j0;     // fitness index of each tie
        const long long* toff = g.tie_off + g.tp_row0[tp] + j0;  // its row's population offset
        const InstDesc d = a.desc[g.row_exec[g.tp_row0[tp]]];  // dim, objective and problem of every tie
        const float* o = a.shift + d.shift_off;
        const float* Rr = a.rot + d.rot_off;  // R rows [dim][dpad]
        const int nchunk = (d.dim + kRc - 1) / kRc;
        auto stage = [&](int ch) {  // R[r][ch * 16 ..] for every row r < dim into stage ch % kRing
            if (ch < nchunk) {
                float* dst = sR + (size_t)(ch % kRing) * kVec * kRcs;
                const int c0 = ch * kRc;
                for (int e2 = tid; e2 < d.dim * (kRc / 4); e2 += kSelThreads) {
                    const int rr = e2 >> 2, c = c0 + 4 * (e2 & 3);
                    const bool in = c < d.dpad;
                    cp_async16z(dst + rr * kRcs + 4 * (e2 & 3), Rr + (size_t)rr * d.dpad + (in ? c : 0),
                                in ? 16 : 0);
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");  // one group per stage, empty past the end
        };
        for (int ch = 0; ch < kRing - 1; ++ch) stage(ch);
        {  // x - o and u - x of every tie, float4 at a time (pad columns of x, u and o are zero)
            const int f4 = d.dpad >> 2;
            for (int e2 = tid; e2 < nb * f4; e2 += kSelThreads) {
                const int q = e2 / f4, c = 4 * (e2 - q * f4);
                const long long off = toff[q];
                const float4 x4 = *reinterpret_cast<const float4*>(a.pop + off + c);
                const float4 u4 = __ldg(reinterpret_cast<const float4*>(g.uscr + off + c));
                const float4 o4 = __ldg(reinterpret_cast<const float4*>(o + c));
                *reinterpret_cast<float4*>(vx + q * kVec + c) = make_float4(x4.x - o4.x, x4.y - o4.y, x4.z - o4.z,
                                                                            x4.w - o4.w);
                *reinterpret_cast<float4*>(vl + q * kVec + c) = make_float4(u4.x - x4.x, u4.y - x4.y, u4.z - x4.z,
                                                                            u4.w - x4.w);
            }
        }
        // thread (rows r and r + half, group h): half = vrow / 2 threads per group, vrow = the rows
        // rounded up to a power of two (64 .. 256), G = 512 / half groups (4 .. 16); group h takes
        // ties h, h + G, ... of the chunk (at most four), so narrow problems keep every thread busy
        // and each shared-memory load of x - o or u - x feeds two rows
        int lg = 6;
        while ((1 << lg) < d.dim) ++lg;
        const int half = 1 << (lg - 1);
        const int G = kSelThreads / half;
        const int r = tid & (half - 1), h = tid / half;  // h is uniform over a warp (half >= 32)
        const bool row1 = r + half < d.dim;
        float az[kTieBatch / 4][2], adz[kTieBatch / 4][2];
#pragma unroll
        for (int q = 0; q < kTieBatch / 4; ++q) az[q][0] = az[q][1] = adz[q][0] = adz[q][1] = 0.f;
        const int mine = (nb - h + G - 1) / G;  // ties of this group
        for (int ch = 0; ch < nchunk; ++ch) {
            stage(ch + kRing - 1);  // the stage read at ch - 1 is free: every thread passed the barrier after it
            asm volatile("cp.async.wait_group %0;" ::"n"(kRing - 1) : "memory");  // stage ch has landed
            __syncthreads();
            if (r < d.dim) {  // (rows r + half >= D compute from stale stage rows; they are not stored)
                const float* rc0 = sR + (size_t)(ch % kRing) * kVec * kRcs + r * kRcs;
                const float* rc1 = rc0 + half * kRcs;
                const int c0 = ch * kRc;
                const int cend = min(kRc, d.dim - c0);
                if (cend == kRc) {  // four float4 steps, k ascending within each
#pragma unroll
                    for (int c4 = 0; c4 < kRc / 4; ++c4) {
                        const float4 ra = *reinterpret_cast<const float4*>(rc0 + 4 * c4);
                        const float4 rb = *reinterpret_cast<const float4*>(rc1 + 4 * c4);
#pragma unroll
                        for (int j = 0; j < kTieBatch / 4; ++j) {
                            if (j < mine) {
                                const int q = h + G * j;
                                const float4 x4 = *reinterpret_cast<const float4*>(vx + q * kVec + c0 + 4 * c4);
                                const float4 l4 = *reinterpret_cast<const float4*>(vl + q * kVec + c0 + 4 * c4);
                                az[j][0] = fmaf(ra.x, x4.x, az[j][0]);
                                az[j][1] = fmaf(rb.x, x4.x, az[j][1]);
                                adz[j][0] = fmaf(ra.x, l4.x, adz[j][0]);
                                adz[j][1] = fmaf(rb.x, l4.x, adz[j][1]);
                                az[j][0] = fmaf(ra.y, x4.y, az[j][0]);
                                az[j][1] = fmaf(rb.y, x4.y, az[j][1]);
                                adz[j][0] = fmaf(ra.y, l4.y, adz[j][0]);
                                adz[j][1] = fmaf(rb.y, l4.y, adz[j][1]);
                                az[j][0] = fmaf(ra.z, x4.z, az[j][0]);
                                az[j][1] = fmaf(rb.z, x4.z, az[j][1]);
                                adz[j][0] = fmaf(ra.z, l4.z, adz[j][0]);
                                adz[j][1] = fmaf(rb.z, l4.z, adz[j][1]);
                                az[j][0] = fmaf(ra.w, x4.w, az[j][0]);
                                az[j][1] = fmaf(rb.w, x4.w, az[j][1]);
                                adz[j][0] = fmaf(ra.w, l4.w, adz[j][0]);
                                adz[j][1] = fmaf(rb.w, l4.w, adz[j][1]);
                            }
                        }
                    }
                } else {  // the last, partial chunk: one column at a time
                    for (int cc = 0; cc < cend; ++cc) {
                        const float ra = rc0[cc], rb = rc1[cc];
#pragma unroll
                        for (int j = 0; j < kTieBatch / 4; ++j) {
                            if (j < mine) {
                                const int q = h + G * j;
                                const float xk = vx[q * kVec + c0 + cc], lk = vl[q * kVec + c0 + cc];
                                az[j][0] = fmaf(ra, xk, az[j][0]);
                                az[j][1] = fmaf(rb, xk, az[j][1]);
                                adz[j][0] = fmaf(ra, lk, adz[j][0]);
                                adz[j][1] = fmaf(rb, lk, adz[j][1]);
                            }
                        }
                    }
                }
            }
            __syncthreads();  // the stage is refilled kRing - 1 chunks later
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");  // only empty groups remain
        if (r < d.dim) {  // every thread has read vx / vl: z and dz replace them
#pragma unroll
            for (int j = 0; j < kTieBatch / 4; ++j) {
                if (j < mine) {
                    const int q = h + G * j;
                    vx[q * kVec + r] = az[j][0];
                    vl[q * kVec + r] = adz[j][0];
                    if (row1) {
                        vx[q * kVec + r + half] = az[j][1];
                        vl[q * kVec + r + half] = adz[j][1];
                    }
                }
            }
        }
        __syncthreads();
        if (warp < nb) {  // warp per tie: decide and commit
            const long long off = toff[warp];
            const int fidx = tfid[warp];
            bool diff = false;  // every load issued: no short circuit
            for (int c = lane; c < d.dpad; c += 32) diff |= g.uscr[off + c] != a.pop[off + c];
            const float fx = a.fit[fidx];
            bool take;
            float fn;
            if (!__any_sync(kFull, diff)) {  // a trial identical to its target: accepted as it is
                take = true;
                fn = fx;
            } else {
                const float df = warp_diff(d.obj, d.dim, vx + warp * kVec, vl + warp * kVec);
                take = df <= 0.0f;
                fn = fx + df;
            }
            if (take) {
                for (int c = 4 * lane; c < d.dpad; c += 128)
                    *reinterpret_cast<float4*>(a.pop + off + c) = *reinterpret_cast<const float4*>(g.uscr + off + c);
                if (lane == 0) a.fit[fidx] = fn;
            }
        }
        __syncthreads();  // the buffers and the chunk record are reused
    }
}

// ---------------------------------------------------------- k_tc_ties_wide
constexpr int kWThreads = 256;                // threads of k_tc_ties_wide
constexpr int kWRows = 2;                     // consecutive rows of z per thread
constexpr int kWGroup = kWThreads * kWRows;   // rows of z per work item
constexpr int kWMaxTies = 8;                  // near ties of one problem per chunk at most
constexpr int kWCk = 16;                      // columns of R^T per stage
constexpr int kWStages = 3;                   // stages of the cp.async ring
constexpr int kWStageR = kWCk * kWGroup;      // floats of R^T per stage (32 KB)
constexpr int kWStageV = 2 * kWMaxTies * kWCk + kWCk;  // x and u of every tie, then o, for the stage's columns
constexpr int kWStage = kWStageR + kWStageV;  // floats per stage
static_assert(kWStage % 4 == 0, "stages start 16-byte aligned");
static_assert(kWRows == 2, "the sweep loads two rows of R^T per column as a float2");

struct TieWArgs {
    StepArgs a;
    const int* row_exec;      // operand row -> executor
    int n_tp;                 // problems on this path
    const int* tp_row0;       // per problem: start of its tie list
    const int* tie_cnt;       // per problem: near ties listed by the GEMM kernel
    const int* tie_list;      // fitness index of each near tie, by problem
    const long long* tie_off; // population offset of each near tie's row, by problem
    int* item_ctr;            // work items handed out (zeroed by k_tc_rank)
    int* done;                // per chunk (at its first list slot): row groups finished; the last one resets it
    float* zs;                // [list slot][2][vs]: z and dz of each near tie
    const float* uscr;        // trial rows (population layout)
    int vs;                   // floats per vector of z: round_up(the widest D_pad, 4)
    int ngmax;                // row groups of the widest problem
    unsigned long long* tie_total;  // near ties decided, summed over generations (block 0 adds)
};

// Near ties of problems wider than 256, for the four-kernel generation whose
// GEMM kernel is k_rot_tc.  A work item is (chunk of up to kWMaxTies ties of
// one problem, group of 512 rows of z).  R^T is streamed 16 columns at a time
// through a 3-stage cp.async ring, together with those columns of x, u and o
// of every tie of the chunk (x - o and u - x are formed once per stage); a
// thread owns two consecutive rows and forms their z = R (x - o) and
// dz = R (u - x) for every tie in FP32, a float2 of R^T per column against a
// float4 of x - o (and u - x) per tie and four columns.
// Every fma chain runs in ascending k like every other FP32 rotation; the
// columns past D are zero in all three operands (fma(0, 0, acc) == acc for an
// accumulator that starts at +0), so the results are bit-identical to a plain
// loop over k < D.  The stage loop is instantiated for 1, 2, 4 and 8 ties.  The rows go to a
// global scratch; the CTA that finishes a chunk's last row group (a counter
// per chunk) reads z and dz back through L2, and a warp per tie forms the
// FP32 difference form, decides and commits.  A trial identical to its
// target is accepted as it is.  Splitting the rows over CTAs keeps every SM
// streaming R even when a generation has few ties.
// The stage loop of k_tc_ties_wide for NB ties (a power of two >= the
// chunk's ties; the rest are zero-filled and their rows not stored): no
// branch inside, so the loads of a step are issued ahead of its fmas.
template <int NB, typename Issue>
__device__ __forceinline__ void wide_sweep(int nst, int nb, const float* ring, float* sx, float* sl, Issue& issue,
                                           float* zs, int slot0, int vs, int r0, int dim) {
    const int tid = threadIdx.x;
    float az[NB][kWRows], adz[NB][kWRows];
#pragma unroll
    for (int t = 0; t < NB; ++t)
#pragma unroll
        for (int j = 0; j < kWRows; ++j) az[t][j] = adz[t][j] = 0.f;
    for (int st = 0; st < nst; ++st) {
        issue(st + kWStages - 1);  // the stage read at st - 1 is free: every thread passed the barrier after it
        asm volatile("cp.async.wait_group %0;" ::"n"(kWStages - 1) : "memory");  // stage st has landed
        __syncthreads();
        const float* buf = ring + (size_t)(st % kWStages) * kWStage;
        if (tid < kWMaxTies * kWCk) {  // x - o and u - x of the stage's columns, a thread per (tie, column)
            const int t = tid / kWCk, k = tid - t * kWCk;
            const float* v = buf + kWStageR;
            const float x = v[t * kWCk + k], u = v[kWMaxTies * kWCk + t * kWCk + k], oo = v[2 * kWMaxTies * kWCk + k];
            sx[t * kWCk + k] = x - oo;
            sl[t * kWCk + k] = u - x;
        }
        __syncthreads();
#pragma unroll
        for (int c4 = 0; c4 < kWCk / 4; ++c4) {
            float rt[4][kWRows];  // R^T[c][this thread's rows] for the four columns c of the step
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 r2 = *reinterpret_cast<const float2*>(buf + (4 * c4 + k) * kWGroup + kWRows * tid);
                rt[k][0] = r2.x;
                rt[k][1] = r2.y;
            }
#pragma unroll
            for (int t = 0; t < NB; ++t) {
                const float4 x4 = *reinterpret_cast<const float4*>(sx + t * kWCk + 4 * c4);
                const float4 l4 = *reinterpret_cast<const float4*>(sl + t * kWCk + 4 * c4);
                const float xk[4] = {x4.x, x4.y, x4.z, x4.w}, lk[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
#pragma unroll
                    for (int j = 0; j < kWRows; ++j) {
                        az[t][j] = fmaf(rt[k][j], xk[k], az[t][j]);
                        adz[t][j] = fmaf(rt[k][j], lk[k], adz[t][j]);
                    }
                }
            }
        }
        __syncthreads();  // the stage is refilled kWStages - 1 steps later; sx, sl at the next step
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // only empty groups remain
    if (r0 < dim) {
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            if (t < nb) {
                float* zt = zs + (size_t)(slot0 + t) * 2 * vs + r0;
                *reinterpret_cast<float2*>(zt) = make_float2(az[t][0], az[t][1]);
                *reinterpret_cast<float2*>(zt + vs) = make_float2(adz[t][0], adz[t][1]);
            }
        }
    }
}

__global__ void __launch_bounds__(kWThreads, 2) k_tc_ties_wide(TieWArgs g) {
    extern __shared__ uint8_t smraw[];
    __shared__ int tp_s, j0_s, rg_s, bsz_s, last_s, ncum_s[kMaxTpSmem + 1];
    __shared__ __align__(16) float sx[kWMaxTies * kWCk], sl[kWMaxTies * kWCk];  // x - o, u - x of the stage
    float* ring = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 15) & ~(uintptr_t)15);
    const StepArgs& a = g.a;
    const int vs = g.vs;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto groups = [&](int tp) { return (a.desc[g.row_exec[g.tp_row0[tp]]].dim + kWGroup - 1) / kWGroup; };
    if (tid == 0) {  // chunk size: about one round of items over the grid, 1 .. kWMaxTies ties
        long long total = 0;
        for (int q = 0; q < g.n_tp; ++q) total += g.tie_cnt[q];
        const long long work = total * g.ngmax;  // (tie, row group) pairs
        const long long rounds = max(1LL, (work + (long long)gridDim.x * kWMaxTies - 1) / ((long long)gridDim.x * kWMaxTies));
        const long long per = (long long)gridDim.x * rounds;
        bsz_s = (int)min((long long)kWMaxTies, max(1LL, (work + per - 1) / per));
        if (blockIdx.x == 0) atomicAdd(g.tie_total, (unsigned long long)total);
    }
    __syncthreads();
    const int bsz = bsz_s;
    const bool cum_smem = g.n_tp <= kMaxTpSmem;  // items per problem, summed in problem order
    if (cum_smem) {
        for (int q = tid; q < g.n_tp; q += blockDim.x) ncum_s[q + 1] = (g.tie_cnt[q] + bsz - 1) / bsz * groups(q);
        __syncthreads();
        if (tid == 0) {
            ncum_s[0] = 0;
            for (int q = 0; q < g.n_tp; ++q) ncum_s[q + 1] += ncum_s[q];
        }
        __syncthreads();
    }
    for (;;) {
        if (tid == 0) {  // item w -> (problem, first tie of the chunk, row group)
            const int w = atomicAdd(g.item_ctr, 1);
            int tp = -1, e = 0;
            if (cum_smem) {
                if (w < ncum_s[g.n_tp]) {
                    int lo = 0, hi = g.n_tp - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (ncum_s[mid] <= w) lo = mid;
                        else hi = mid - 1;
                    }
                    tp = lo;
                    e = w - ncum_s[lo];
                }
            } else {
                int acc = 0;
                for (int q = 0; q < g.n_tp; ++q) {
                    const int n = (g.tie_cnt[q] + bsz - 1) / bsz * groups(q);
                    if (w < acc + n) {
                        tp = q;
                        e = w - acc;
                        break;
                    }
                    acc += n;
                }
            }
            tp_s = tp;
            if (tp >= 0) {
                const int ng = groups(tp);
                j0_s = (e / ng) * bsz;
                rg_s = e - (e / ng) * ng;
            }
        }
        __syncthreads();
        const int tp = tp_s;
        if (tp < 0) break;
        const int j0 = j0_s, rg = rg_s;
        const int nb = min(bsz, g.tie_cnt[tp] - j0);
        const int slot0 = g.tp_row0[tp] + j0;  // list slot of the chunk's first tie
        const long long* toff = g.tie_off + slot0;
        const InstDesc d = a.desc[g.row_exec[g.tp_row0[tp]]];
        const int ng = (d.dim + kWGroup - 1) / kWGroup;
        const float* o = a.shift + d.shift_off;
        const float* RT = a.rotT + d.rot_off;  // R^T [dim][dpad]
        const int rbase = rg * kWGroup;        // first row of the item
        const int nst = (d.dim + kWCk - 1) / kWCk;
        // stage st: R^T[c][rbase ..] for its 16 columns c, and x, u, o in those columns;
        // anything past D (columns) or D_pad (rows) is zero-filled
        auto issue = [&](int st) {
            if (st < nst) {
                float* buf = ring + (size_t)(st % kWStages) * kWStage;
                const int c0 = st * kWCk;
                for (int e2 = tid; e2 < kWCk * (kWGroup / 4); e2 += kWThreads) {
                    const int k = e2 / (kWGroup / 4), i4 = 4 * (e2 - k * (kWGroup / 4));
                    const bool ok = c0 + k < d.dim && rbase + i4 < d.dpad;
                    cp_async16z(buf + k * kWGroup + i4, ok ? RT + (size_t)(c0 + k) * d.dpad + rbase + i4 : RT,
                                ok ? 16 : 0);
                }
                if (tid < 2 * kWMaxTies * (kWCk / 4) + kWCk / 4) {  // x, u of each tie, then o: 16 bytes each
                    const int part = tid / (kWMaxTies * (kWCk / 4));  // 0 x, 1 u, 2 o
                    const int rem = tid - part * (kWMaxTies * (kWCk / 4));
                    const int t = rem / (kWCk / 4), col = c0 + 4 * (rem % (kWCk / 4));
                    const bool ok = col < d.dpad && (part == 2 || t < nb);
                    const float* src = part == 2 ? o + col
                                       : (part == 0 ? a.pop : g.uscr) + (ok ? toff[t] : 0) + col;
                    cp_async16z(buf + kWStageR + part * kWMaxTies * kWCk + 4 * rem, ok ? src : o, ok ? 16 : 0);
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");  // one group per stage, empty past the end
        };
        for (int st = 0; st < kWStages - 1; ++st) issue(st);
        const int r0 = rbase + kWRows * tid;  // this thread's first row (rows r0, r0 + 1 < D_pad)
        if (nb <= 1) wide_sweep<1>(nst, nb, ring, sx, sl, issue, g.zs, slot0, vs, r0, d.dim);
        else if (nb <= 2) wide_sweep<2>(nst, nb, ring, sx, sl, issue, g.zs, slot0, vs, r0, d.dim);
        else if (nb <= 4) wide_sweep<4>(nst, nb, ring, sx, sl, issue, g.zs, slot0, vs, r0, d.dim);
        else wide_sweep<8>(nst, nb, ring, sx, sl, issue, g.zs, slot0, vs, r0, d.dim);
        __threadfence();  // this group's rows are visible before the chunk's counter moves
        __syncthreads();
        if (tid == 0) last_s = atomicAdd(&g.done[slot0], 1) == ng - 1;
        __syncthreads();
        if (last_s) {  // every row group of the chunk is in: decide its ties
            __threadfence();
            float* vz = ring;                       // [nb][vs] z, then [nb][vs] dz (over the ring)
            float* vd = ring + (size_t)kWMaxTies * vs;
            const int f4 = d.dpad >> 2;
            for (int e2 = tid; e2 < nb * f4; e2 += kWThreads) {  // through L2 (not L1)
                const int q = e2 / f4, c = 4 * (e2 - q * f4);
                const float* zt = g.zs + (size_t)(slot0 + q) * 2 * vs + c;
                *reinterpret_cast<float4*>(vz + q * vs + c) = __ldcg(reinterpret_cast<const float4*>(zt));
                *reinterpret_cast<float4*>(vd + q * vs + c) = __ldcg(reinterpret_cast<const float4*>(zt + vs));
            }
            __syncthreads();
            for (int t = warp; t < nb; t += kWThreads / 32) {  // a warp per tie
                const long long off = toff[t];
                const int fidx = g.tie_list[slot0 + t];
                bool diff = false;  // every load issued: no short circuit
                for (int c = lane; c < d.dpad; c += 32) diff |= g.uscr[off + c] != a.pop[off + c];
                const float fx = a.fit[fidx];
                bool take;
                float fn;
                if (!__any_sync(kFull, diff)) {  // a trial identical to its target: accepted as it is
                    take = true;
                    fn = fx;
                } else {
                    const float df = warp_diff(d.obj, d.dim, vz + t * vs, vd + t * vs);
                    take = df <= 0.0f;
                    fn = fx + df;
                }
                if (take) {
                    for (int c = 4 * lane; c < d.dpad; c += 128)
                        *reinterpret_cast<float4*>(a.pop + off + c) =
                            *reinterpret_cast<const float4*>(g.uscr + off + c);
                    if (lane == 0) a.fit[fidx] = fn;
                }
            }
            if (tid == 0) g.done[slot0] = 0;  // ready for the next generation
        }
        __syncthreads();  // the ring and the item record are reused
    }
}

// best and the pbest pool of every tensor-core executor (block per executor;
// best alone, by an argmin, when the strategy draws no pbest);
// block 0 also zeroes the tile counter of the k_tc_sel launch that follows.
// With trec, a thread per row then writes the row's draw record for
// k_tc_trial2 (4 int4: base and difference indices as 16-bit pairs, j_rand
// and the exponential start, K, the row index with the strategy bits and a
// valid bit, the population offset, F, the CR threshold, the Philox stream,
// D and D_pad, the shift offset, the fitness index); rows of an invalid theta
// get valid = 0.
__global__ void __launch_bounds__(256, 8) k_tc_rank(StepArgs a, const int* __restrict__ execs, int* topk_all, int* next_tile, int* chunk_ctr,
                          int* tie_cnt, int n_tp, int4* trec) {
    if (blockIdx.x == 0) {  // the queues of k_tc_sel and k_tc_ties2 of this generation
        if (threadIdx.x == 0) *next_tile = *chunk_ctr = 0;
        for (int q = threadIdx.x; q < n_tp; q += blockDim.x) tie_cnt[q] = 0;
    }
    const int k = execs[blockIdx.x];
    const InstDesc d = a.desc[k];
    const Strat s = load_strat(a.theta + 6 * k, d.np);
    if (!s.ok) {
        if (threadIdx.x == 0) set_status(a.status, 1);
        if (trec)
            for (int i = threadIdx.x; i < d.np; i += blockDim.x) {
                int4* q = trec + 4 * (size_t)(d.tc_row + i);
                q[0] = make_int4(0, 0, 0, 0);
                q[1] = make_int4(0, 0, 0, i);
                q[2] = make_int4(0, 0, 0, 0);
                q[3] = make_int4(d.stream, d.dim | (d.dpad << 16), d.shift_off, d.fit_off + i);
            }
        return;
    }
    int* topk = topk_all + d.fit_off;
    __shared__ int red[64];
    if (s.uses_pbest()) {
        block_topk_staged(a.fit + d.fit_off, d.np, d.kp, topk);
    } else {  // best alone, in topk[0]: such a strategy never uses the pool entry indiv_setup reads
        const int b = block_argmin(a.fit + d.fit_off, d.np, red);
        if (threadIdx.x == 0) topk[0] = b;
    }
    if (!trec) return;
    __syncthreads();  // the pool (global memory) is visible to the whole block
    const int best = topk[0];
    const uint32_t epoch = a.epoch_dev ? *a.epoch_dev : a.epoch;
    const int pack = s.cs | (s.dn << 4) | ((s.bl != s.br ? 1 : 0) << 8) | (1 << 12);
    for (int i = threadIdx.x; i < d.np; i += blockDim.x) {
        const Ctr c = make_ctr(a.key, (uint32_t)d.stream, a.gen0, (uint32_t)i, epoch);
        Indiv v;
        indiv_setup(s, c, i, d.np, d.dim, d.kp, topk, best, v);
        int pm[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            pm[2 * q] = q < s.dn ? diff_plus(v, s.a, q) : 0;
            pm[2 * q + 1] = q < s.dn ? diff_minus(v, s.a, q) : 0;
        }
        int4* q = trec + 4 * (size_t)(d.tc_row + i);
        q[0] = make_int4(v.ibl | (v.ibr << 16), pm[0] | (pm[1] << 16), pm[2] | (pm[3] << 16), pm[4] | (pm[5] << 16));
        q[1] = make_int4(pm[6] | (pm[7] << 16), v.jrand | (v.nstart << 16), (int)v.kraw, i | (pack << 16));
        q[2] = make_int4((int)(uint32_t)d.pop_off, (int)(d.pop_off >> 32), __float_as_int(s.F), (int)s.cri);
        q[3] = make_int4(d.stream, d.dim | (d.dpad << 16), d.shift_off, d.fit_off + i);
    }
}

size_t sel_smem(int kt) { return 1024 + kASize + kPartSize + (size_t)kt * kBT; }
constexpr size_t kTieSmem = 16 + kTie2Size;
// the ring, or (for the chunk's decision) z and dz of kWMaxTies ties, whichever is larger
size_t wide_smem(int vs) {
    return 16 + std::max((size_t)kWStages * kWStage, (size_t)2 * kWMaxTies * vs) * sizeof(float);
}
int wide_vs(int max_dpad) { return (max_dpad + 3) & ~3; }

}  // namespace

bool tc_fused_fits(int kp) { return kp <= kMaxKt * kBK && sel_smem(kp / kBK) <= 227 * 1024; }

int tc_ties_wide_ctas(int max_dpad) {
    const size_t smem = wide_smem(wide_vs(max_dpad));
    if (cudaFuncSetAttribute(k_tc_ties_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tc_ties_wide, kWThreads, smem) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
        return 0;
    return per_sm * sms;
}

cudaError_t launch_tc_trial_rows32(const StepArgs& a, const TcPlan& p, void* aq, const int4* trec, cudaStream_t st) {
    k_tc_trial2<<<(p.n_rows + kTRows - 1) / kTRows, kTThreads, 0, st>>>(a, p.row_exec, p.n_rows, p.topk_all, p.uscr,
                                                                       static_cast<uint8_t*>(aq), p.kp, trec);
    return cudaGetLastError();
}

cudaError_t launch_tc_rank(const StepArgs& a, const TcPlan& p, int4* trec, cudaStream_t st) {
    k_tc_rank<<<p.n_exec, 256, 0, st>>>(a, p.execs, p.topk_all, p.next_tile, p.chunk_ctr, p.tie_cnt, p.n_tp,
                                        trec);
    return cudaGetLastError();
}

cudaError_t launch_tc_ties_batched(const StepArgs& a, const TcPlan& p, cudaStream_t st) {
    cudaError_t e;
    if (p.max_dpad > kVec) {
        TieWArgs tw;
        tw.a = a;
        tw.row_exec = p.row_exec;
        tw.n_tp = p.n_tp;
        tw.tp_row0 = p.tp_row0;
        tw.tie_cnt = p.tie_cnt;
        tw.tie_list = p.tie_list;
        tw.tie_off = p.tie_off;
        tw.item_ctr = p.chunk_ctr;
        tw.done = p.tie_done;
        tw.zs = p.tie_zs;
        tw.uscr = p.uscr;
        tw.tie_total = p.tie_total;
        tw.vs = wide_vs(p.max_dpad);
        tw.ngmax = (p.max_dpad + kWGroup - 1) / kWGroup;
        const size_t smem = wide_smem(tw.vs);
        e = cudaFuncSetAttribute(k_tc_ties_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tc_ties_wide<<<p.wide_ctas, kWThreads, smem, st>>>(tw);
        return cudaGetLastError();
    }
    TieArgs ta;
    ta.a = a;
    ta.row_exec = p.row_exec;
    ta.n_tp = p.n_tp;
    ta.tp_row0 = p.tp_row0;
    ta.tie_cnt = p.tie_cnt;
    ta.tie_list = p.tie_list;
    ta.tie_off = p.tie_off;
    ta.chunk_ctr = p.chunk_ctr;
    ta.uscr = p.uscr;
    ta.tie_total = p.tie_total;
    e = cudaFuncSetAttribute(k_tc_ties2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTieSmem);
    if (e != cudaSuccess) return e;
    k_tc_ties2<<<2 * p.gen_ctas, kSelThreads, kTieSmem, st>>>(ta);
    return cudaGetLastError();
}

cudaError_t launch_tc_fused_generation(const StepArgs& a, const TcPlan& p, cudaStream_t st, cudaEvent_t* ev) {
    if (ev) cudaEventRecord(ev[0], st);
    // plan mode 1: the draws go with the ranking, and k_tc_trial2 reads them
    int4* trec = p.fused == 1 ? p.trial_rec : nullptr;
    k_tc_rank<<<p.n_exec, 256, 0, st>>>(a, p.execs, p.topk_all, p.next_tile, p.chunk_ctr, p.tie_cnt, p.n_tp, trec);
    if (ev) cudaEventRecord(ev[1], st);
    cudaError_t e;
    if (p.fused == 2) {  // operands wider than 256: warp-per-row trials, k_rot_tc selecting, row-split ties
        e = launch_tc_trial_rows(a, p, st);
        if (e != cudaSuccess) return e;
        if (ev) cudaEventRecord(ev[2], st);
        e = launch_rot_tc_select(a, p, st);
        if (e != cudaSuccess) return e;
        if (ev) cudaEventRecord(ev[3], st);
        e = launch_tc_ties_batched(a, p, st);
        if (e != cudaSuccess) return e;
        if (ev) cudaEventRecord(ev[4], st);
        return cudaGetLastError();
    }
    k_tc_trial2<<<(p.n_rows + kTRows - 1) / kTRows, kTThreads, 0, st>>>(a, p.row_exec, p.n_rows, p.topk_all, p.uscr,
                                                                       static_cast<uint8_t*>(p.aq), p.kp, trec);
    if (ev) cudaEventRecord(ev[2], st);
    {
        SelArgs g;
        g.a = a;
        g.tiles = p.tiles;
        g.n_tiles = p.n_tiles;
        g.next_tile = p.next_tile;
        g.prob_tp = p.prob_tp;
        g.tp_row0 = p.tp_row0;
        g.tie_cnt = p.tie_cnt;
        g.tie_list = p.tie_list;
        g.tie_off = p.tie_off;
        g.row_exec = p.row_exec;
        g.brow = p.brow;
        g.uscr = p.uscr;
        g.kt = p.kp / kBK;
        g.tmeta = p.tmeta;
        g.trec = trec;
        const size_t smem = sel_smem(g.kt);
        e = cudaFuncSetAttribute(k_tc_sel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int grid = p.n_tiles < p.gen_ctas ? p.n_tiles : p.gen_ctas;
        k_tc_sel<<<grid, kSelThreads + 32, smem, st>>>(p.mapA, p.mapB, g);
    }
    if (ev) cudaEventRecord(ev[3], st);
    e = launch_tc_ties_batched(a, p, st);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[4], st);
    return cudaGetLastError();
}

}  // namespace metade
