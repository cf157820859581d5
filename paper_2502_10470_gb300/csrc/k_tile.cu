// k_tile.cu -- batched path for 32 < D <= 128: k_fused_tile.
//
// One CTA per executor runs all fused generations.  Each generation walks
// the population in tiles of kT individuals:
//   trial      thread per individual for the draws (a record in shared
//              memory), then (chunk, individual) work items for mutation,
//              crossover and clip; the FP32 trial row goes to the scratch
//              population, d = u - o to a k-major tile dT[k][t]
//   rotation   Z = d R^T by 4x4 register blocks, R^T resident in shared memory
//   objective  four lanes per individual over its Z row
// then selection: the clear cases by a thread per individual, the near ties
// kT / 2 at a time through the same GEMM (x - o and u - x as column pairs)
// and the difference forms, and one coalesced pass copying accepted rows.
#include "block.cuh"
#include "group_obj.cuh"
#include "internal.h"

namespace metade {

namespace {
constexpr int kT = 64;        // individuals per tile
constexpr int kTP = kT + 4;   // k-major row length of dT (float4 aligned)
constexpr int kRec = 14;      // draw record fields, stored field-major (recs[field * kT + t]: no bank conflicts)
static_assert(kRec <= 36, "the draw records alias Z, whose rows are at least 36 floats long");

// Z row stride: at least max_dpad and 4 (mod 32), so the eight 4-lane groups
// of a warp that read 4 consecutive rows of 8 different Z rows hit distinct banks.
__host__ __device__ constexpr int tile_zp(int max_dpad) { return max_dpad + ((4 - max_dpad) % 32 + 32) % 32; }
}  // namespace

// Z[t][r] = sum_k dT[k][t] R^T[k][r] for the kT columns of dT: every thread
// owns 4x4 blocks of Z and reads one float4 of dT and one of R^T per k (16
// FMAs per two loads); k ascends, so each z is the fma chain of every other
// rotation in the library.
__device__ __forceinline__ void tile_gemm(const float* dT, const float* RT, float* Z, int dim, int nbr, int dp,
                                          int zp) {
    constexpr int nbt = kT / 4;
    for (int blk = threadIdx.x; blk < nbt * nbr; blk += blockDim.x) {
        const int tx = blk % nbt, ty = blk / nbt;
        float acc[4][4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
        const float* pa = dT + 4 * tx;
        const float* pr = RT + 4 * ty;
        for (int kk = 0; kk < dim; ++kk) {
            const float4 av = *reinterpret_cast<const float4*>(pa + (size_t)kk * kTP);
            const float4 rv = *reinterpret_cast<const float4*>(pr + (size_t)kk * dp);
            const float ar[4] = {av.x, av.y, av.z, av.w}, rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(rr[q], ar[p], acc[p][q]);
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
            *reinterpret_cast<float4*>(Z + (size_t)(4 * tx + p) * zp + 4 * ty) =
                make_float4(acc[p][0], acc[p][1], acc[p][2], acc[p][3]);
    }
}

// R^T streamed from global memory (executors whose R^T does not stay in
// shared memory, 128 < D_pad <= 256): kKC rows of R^T at a time go through a
// double-buffered cp.async stage; every thread keeps the accumulators of up
// to four 4x4 blocks of Z (the same tx, ty = ty0 + 16 j) in registers across
// the chunks, so the fma chain of each z is the same as above.  256 threads.
// Z may alias dT: it is written after the last chunk's barrier.
constexpr int kKC = 16;

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void stage_rt(float* dst, const float* __restrict__ gRT, int k0, int kn, int dp) {
    const int n4 = kn * (dp >> 2);
    const float* src = gRT + (size_t)k0 * dp;
    for (int e = threadIdx.x; e < n4; e += blockDim.x) cp_async16(dst + 4 * e, src + 4 * e);
}

__device__ __forceinline__ void tile_gemm_stream(const float* dT, const float* __restrict__ gRT, float* rbuf, float* Z,
                                                 int dim, int nbr, int dp, int zp) {
    constexpr int nbt = kT / 4;                  // 16 column blocks of the tile
    const int tid = threadIdx.x;
    const int tx = tid % nbt, ty0 = tid / nbt;   // 256 threads: ty0 < 16, blocks ty0 + 16 j, j < 4
    const int nj = ty0 < nbr ? (nbr - ty0 + 15) / 16 : 0;
    float acc[4][4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[j][p][q] = 0.f;
    const int nch = (dim + kKC - 1) / kKC;
    stage_rt(rbuf, gRT, 0, min(kKC, dim), dp);
    cp_async_commit();
    const float* pa = dT + 4 * tx;
    for (int ch = 0; ch < nch; ++ch) {
        if (ch + 1 < nch) {
            stage_rt(rbuf + ((ch + 1) & 1) * kKC * dp, gRT, (ch + 1) * kKC, min(kKC, dim - (ch + 1) * kKC), dp);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float* rb = rbuf + (ch & 1) * kKC * dp + 4 * ty0;
        const int k0 = ch * kKC, kn = min(kKC, dim - k0);
        for (int kk = 0; kk < kn; ++kk) {
            const float4 av = *reinterpret_cast<const float4*>(pa + (size_t)(k0 + kk) * kTP);
            const float ar[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j < nj) {
                    const float4 rv = *reinterpret_cast<const float4*>(rb + (size_t)kk * dp + 64 * j);
                    const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[j][p][q] = fmaf(rr[q], ar[p], acc[j][p][q]);
                }
            }
        }
        __syncthreads();  // every thread is done with this buffer (and, after the last chunk, with dT)
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (j < nj) {
            const int ty = ty0 + 16 * j;
#pragma unroll
            for (int p = 0; p < 4; ++p)
                *reinterpret_cast<float4*>(Z + (size_t)(4 * tx + p) * zp + 4 * ty) =
                    make_float4(acc[j][p][0], acc[j][p][1], acc[j][p][2], acc[j][p][3]);
        }
    }
}

// Shared words before R^T: f, fu, ranks/flags, tie list, 64 reduction words,
// the tie count and kT / 2 identity flags; a multiple of 4 (float4 alignment).
__host__ __device__ constexpr int tile_header_words(int max_np) { return (4 * max_np + 64 + 1 + kT / 2 + 3) & ~3; }

// Streamed layout: the dT / Z union (dT is dead when Z is written).
__host__ __device__ constexpr int tile_dz_words(int max_dpad) {
    return max_dpad * kTP > kT * tile_zp(max_dpad) ? max_dpad * kTP : kT * tile_zp(max_dpad);
}

// RS: R^T resident in shared memory (D_pad <= 128); otherwise streamed.
// The near ties' difference forms, out of line: every objective's form inlined
// would spread the fused loop's code (measured 3.6% slower).
__device__ __noinline__ float tile_diff_cold(int obj, const float* z, const float* dz, int s, int dim) {
    return group_diff_row<4>(obj, z, dz, s, dim);
}

template <bool RS>
__global__ void __launch_bounds__(256, 2) k_fused_tile(StepArgs a, const int* __restrict__ work, int n_work,
                                                       float* uscr, int max_np, int max_dpad) {
    extern __shared__ __align__(16) float sm[];
    const int tid = threadIdx.x, nt = blockDim.x;  // 128 or 256 threads
    float* f = sm;
    float* fu = f + max_np;
    int* topk = reinterpret_cast<int*>(fu + max_np);               // pbest ranks; selection: accept flags
    int* tl = topk + max_np;                                       // near-tie list
    int* red = tl + max_np;                                        // 64 words (block reductions)
    int* ntie = red + 64;                                          // tie count, then kT / 2 identity flags
    int* idf = ntie + 1;
    const int zp = tile_zp(max_dpad);                              // Z row length
    float* RT;    // resident: [dim][dp]
    float* dT;    // [dp][kTP]
    float* Z;     // [kT][zp]
    float* rbuf;  // streamed: 2 x [kKC][dp]
    int* recs;    // [kRec][kT]
    if (RS) {
        RT = sm + tile_header_words(max_np);
        dT = RT + (size_t)max_dpad * max_dpad;
        Z = dT + (size_t)max_dpad * kTP;
        rbuf = nullptr;
        recs = reinterpret_cast<int*>(Z);  // dead before Z is written
    } else {
        RT = nullptr;
        dT = sm + tile_header_words(max_np);
        Z = dT;                            // written after the GEMM's last read of dT
        rbuf = dT + tile_dz_words(max_dpad);
        recs = reinterpret_cast<int*>(rbuf + 2 * kKC * max_dpad);
    }
    int* acc = topk;
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const int k = work[w];
        const InstDesc d = a.desc[k];
        const Strat st = load_strat(a.theta + 6 * k, d.np);
        if (!st.ok) {
            if (tid == 0) set_status(a.status, 1);
            continue;
        }
        const int np = d.np, dim = d.dim, dp = d.dpad, nbr = dp >> 2;
        const float band = tie_band(dim);
        const uint32_t epoch = a.epoch_dev ? *a.epoch_dev : a.epoch;
        float* X = a.pop + d.pop_off;
        float* Ug = uscr + d.pop_off;
        const float* o = a.shift + d.shift_off;
        const float* gRT = a.rotT + d.rot_off;
        if (RS)
            for (int e = tid; e < dim * (dp >> 2); e += nt)
                reinterpret_cast<float4*>(RT)[e] = reinterpret_cast<const float4*>(gRT)[e];
        for (int i = tid; i < np; i += nt) f[i] = a.fit[d.fit_off + i];
        __syncthreads();
        const bool pb = st.uses_pbest();
        for (int g = 0; g < a.n_gens; ++g) {
            const uint32_t gen = a.gen0 + (uint32_t)g;
            int best;
            if (pb) {
                block_topk(f, np, d.kp, topk);
                __syncthreads();
                best = topk[0];
            } else {
                best = block_argmin(f, np, red);
            }
            for (int t0 = 0; t0 < np; t0 += kT) {
                const int nv = min(kT, np - t0);
                // trial, phase 1: draws of each individual of the tile (thread per individual)
                for (int t = tid; t < kT; t += nt) {
                    int* rec = recs + t;
                    if (t < nv) {
                        const int i = t0 + t;
                        const Ctr c = make_ctr(a.key, (uint32_t)d.stream, gen, (uint32_t)i, epoch);
                        Indiv v;
                        indiv_setup(st, c, i, np, dim, d.kp, pb ? topk : nullptr, best, v);
                        rec[0 * kT] = v.ibl;
                        rec[1 * kT] = v.ibr;
                        rec[2 * kT] = v.jrand;
                        rec[3 * kT] = v.nstart;
                        rec[4 * kT] = st.cs == 2 ? exp_length(c, dim, st.cri) : 0;
                        rec[5 * kT] = (int)v.kraw;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            rec[(6 + 2 * q) * kT] = diff_plus(v, st.a, q);
                            rec[(7 + 2 * q) * kT] = diff_minus(v, st.a, q);
                        }
                    }
                }
                __syncthreads();
                // trial, phase 2: (chunk, individual) items; a warp takes 8
                // individuals x 4 consecutive chunks, so four lanes read 64
                // contiguous bytes of each parent row (two full sectors)
                const int nqb = (nbr + 3) >> 2;
                for (int e = tid; e < nqb * 4 * kT; e += nt) {
                    const int blk = e >> 5, ln = e & 31;
                    const int t = (blk & 7) * 8 + (ln >> 2), q = (blk >> 3) * 4 + (ln & 3), j4 = 4 * q;
                    if (q >= nbr) continue;
                    float* col = dT + (size_t)j4 * kTP + t;
                    if (t >= nv) {
                        col[0] = 0.f; col[kTP] = 0.f; col[2 * kTP] = 0.f; col[3 * kTP] = 0.f;
                        continue;
                    }
                    const int i = t0 + t;
                    const int* rec = recs + t;
                    const float4 av = *reinterpret_cast<const float4*>(X + (long long)rec[0 * kT] * dp + j4);
                    const float4 bv = *reinterpret_cast<const float4*>(X + (long long)rec[1 * kT] * dp + j4);
                    const float4 xv = *reinterpret_cast<const float4*>(X + (long long)i * dp + j4);
                    // every difference-pair row is loaded before any is used, so the
                    // chunk costs one memory round trip whatever dn is
                    float4 pp[4], mm[4];
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        if (qq < st.dn) {
                            pp[qq] = *reinterpret_cast<const float4*>(X + (long long)rec[(6 + 2 * qq) * kT] * dp + j4);
                            mm[qq] = *reinterpret_cast<const float4*>(X + (long long)rec[(7 + 2 * qq) * kT] * dp + j4);
                        }
                    }
                    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        if (qq < st.dn) {
                            sum.x += pp[qq].x - mm[qq].x; sum.y += pp[qq].y - mm[qq].y;
                            sum.z += pp[qq].z - mm[qq].z; sum.w += pp[qq].w - mm[qq].w;
                        }
                    }
                    uint4 wv = make_uint4(0, 0, 0, 0);
                    if (st.cs == 1) {
                        const Ctr c = make_ctr(a.key, (uint32_t)d.stream, gen, (uint32_t)i, epoch);
                        wv = c.slot(4 + (uint32_t)q);
                    }
                    const float F = st.F, K = (float)rec[5 * kT] * (1.0f / 16777216.0f);
                    const bool dir = st.bl != st.br;
                    const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
                    const float x4[4] = {xv.x, xv.y, xv.z, xv.w}, s4[4] = {sum.x, sum.y, sum.z, sum.w};
                    float u4[4];
#pragma unroll
                    for (int tq = 0; tq < 4; ++tq) {
                        const int j = j4 + tq;
                        float vj = a4[tq];
                        if (dir) vj += F * (b4[tq] - a4[tq]);
                        vj += F * s4[tq];
                        float u;
                        if (st.cs == 3) {
                            u = x4[tq] + K * (vj - x4[tq]);
                        } else {
                            bool take;
                            if (st.cs == 1) {
                                take = ((word_of(wv, tq) >> 8) < st.cri) || (j == rec[2 * kT]);
                            } else {
                                int off = j - rec[3 * kT];
                                if (off < 0) off += dim;
                                take = off < rec[4 * kT];
                            }
                            u = take ? vj : x4[tq];
                        }
                        u = fminf(fmaxf(u, a.lo), a.hi);
                        if (j >= dim) u = 0.0f;
                        u4[tq] = u;
                        col[(size_t)tq * kTP] = (j < dim) ? (u - o[j]) : 0.0f;
                    }
                    *reinterpret_cast<float4*>(Ug + (long long)i * dp + j4) = make_float4(u4[0], u4[1], u4[2], u4[3]);
                }
                __syncthreads();
                if (RS) tile_gemm(dT, RT, Z, dim, nbr, dp, zp);
                else tile_gemm_stream(dT, gRT, rbuf, Z, dim, nbr, dp, zp);
                __syncthreads();
                // objective: a group of 4 lanes per individual walks its Z row in
                // blocks of 4 rows (the loop is warp-uniform; rows past nv are zero)
                for (int tb = 0; tb < nv; tb += nt >> 2) {
                    const int t = tb + (tid >> 2), s = tid & 3;
                    const float fv = group_obj_row<4>(d.obj, Z + (size_t)t * zp, s, dim);
                    if (s == 0 && t < nv) fu[t0 + t] = nan_to_inf(fv);
                }
                __syncthreads();
            }
            // selection, pass 1 (thread per individual): decide the clear cases,
            // list the near ties (their order is irrelevant: each is decided alone)
            if (tid == 0) *ntie = 0;
            __syncthreads();
            for (int i = tid; i < np; i += nt) {
                const float fn = fu[i];
                int take = 0;
                if (near_tie(fn, f[i], band)) {
                    tl[atomicAdd(ntie, 1)] = i;
                } else if (fn <= f[i]) {
                    take = 1;
                    f[i] = fn;
                }
                acc[i] = take;
            }
            __syncthreads();
            // near ties, kT / 2 per pass through the tile GEMM: column 2q of dT
            // holds x - o and column 2q + 1 holds u - x of tie q, so Z rows 2q
            // and 2q + 1 are z and dz (the same fma chain as every rotation);
            // then four lanes per tie form f(u) - f(x) by the difference forms
            const int nti = *ntie;
            for (int b0 = 0; b0 < nti; b0 += kT / 2) {
                const int nb = min(kT / 2, nti - b0);
                if (tid < kT / 2) idf[tid] = 0;
                __syncthreads();
                const int nqb = (nbr + 3) >> 2;  // a warp: 8 columns x 4 consecutive chunks (as in the trial)
                for (int e = tid; e < nqb * 4 * kT; e += nt) {
                    const int blk = e >> 5, ln = e & 31;
                    const int c = (blk & 7) * 8 + (ln >> 2), q = (blk >> 3) * 4 + (ln & 3), tt = c >> 1, j4 = 4 * q;
                    if (q >= nbr) continue;
                    float v4[4] = {0.f, 0.f, 0.f, 0.f};
                    if (tt < nb) {
                        const int i = tl[b0 + tt];
                        const float4 xv = *reinterpret_cast<const float4*>(X + (long long)i * dp + j4);
                        const float x4[4] = {xv.x, xv.y, xv.z, xv.w};
                        if (c & 1) {
                            const float4 uv = *reinterpret_cast<const float4*>(Ug + (long long)i * dp + j4);
                            const float u4[4] = {uv.x, uv.y, uv.z, uv.w};
                            bool moved = false;
#pragma unroll
                            for (int tq = 0; tq < 4; ++tq) {
                                if (j4 + tq < dim) {
                                    v4[tq] = u4[tq] - x4[tq];
                                    moved = moved || u4[tq] != x4[tq];
                                }
                            }
                            if (moved) idf[tt] = 1;
                        } else {
#pragma unroll
                            for (int tq = 0; tq < 4; ++tq)
                                if (j4 + tq < dim) v4[tq] = x4[tq] - o[j4 + tq];
                        }
                    }
                    float* col = dT + (size_t)j4 * kTP + c;
                    col[0] = v4[0]; col[kTP] = v4[1]; col[2 * kTP] = v4[2]; col[3 * kTP] = v4[3];
                }
                __syncthreads();
                if (RS) tile_gemm(dT, RT, Z, dim, nbr, dp, zp);
                else tile_gemm_stream(dT, gRT, rbuf, Z, dim, nbr, dp, zp);
                __syncthreads();
                if (tid < 2 * kT) {  // warp-uniform: four lanes for each of the kT / 2 column pairs
                    const int tt = tid >> 2, s = tid & 3;
                    const float* zr = Z + (size_t)(2 * tt) * zp;
                    const float df = tile_diff_cold(d.obj, zr, zr + zp, s, dim);
                    if (s == 0 && tt < nb) {
                        const int i = tl[b0 + tt];
                        if (!idf[tt]) {
                            acc[i] = 1;          // the trial is the target: accepted, f unchanged
                        } else if (df <= 0.0f) {
                            acc[i] = 1;
                            f[i] += df;          // f(x) + (f(u) - f(x)): never above f(x)
                        }
                    }
                }
                __syncthreads();
            }
            // accepted trial rows replace their targets (coalesced float4 copies)
            for (int e = tid; e < np * nbr; e += nt) {
                const int i = e / nbr, q = e - i * nbr;
                if (acc[i])
                    *reinterpret_cast<float4*>(X + (long long)i * dp + 4 * q) =
                        *reinterpret_cast<const float4*>(Ug + (long long)i * dp + 4 * q);
            }
            __syncthreads();
        }
        for (int i = tid; i < np; i += nt) a.fit[d.fit_off + i] = f[i];
        const int b = block_argmin(f, np, red);
        if (tid == 0 && a.best_f) a.best_f[k] = f[b];
        if (tid == 0 && a.best_i) a.best_i[k] = b;
        __syncthreads();
    }
}

size_t fused_smem_tile(int max_np, int max_dpad, int threads, bool rot_smem) {
    (void)threads;
    size_t words = (size_t)tile_header_words(max_np);
    if (rot_smem) {
        words += (size_t)max_dpad * max_dpad;          // R^T
        words += (size_t)max_dpad * kTP;               // dT
        words += (size_t)kT * tile_zp(max_dpad);       // Z (draw records alias it)
    } else {
        words += (size_t)tile_dz_words(max_dpad);      // dT / Z
        words += (size_t)2 * kKC * max_dpad;           // R^T stage
        words += (size_t)kRec * kT;                    // draw records
    }
    return words * sizeof(float);
}

cudaError_t launch_fused_tile(const StepArgs& a, const int* work, int n_work, const FusedPlan& p, float* uscr,
                              cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    if (p.threads != 128 && p.threads != 256) return cudaErrorInvalidValue;
    if (!p.rot_smem && (p.threads != 256 || p.max_dpad > 256)) return cudaErrorInvalidValue;
    auto kern = p.rot_smem ? k_fused_tile<true> : k_fused_tile<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    kern<<<p.grid, p.threads, p.smem, st>>>(a, work, n_work, uscr, p.max_np, p.max_dpad);
    return cudaGetLastError();
}

}  // namespace metade
