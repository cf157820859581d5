// kernels.cu -- CUDA kernels of the MetaDE hot path (sm_103a).
//
//  k_pad_problems   problem table: R rows padded to Dpad, R^T, padded o
//  k_init           Alg. 2 initialisation: population uniform in the box
//  k_eval           shifted-rotated objective of every row, FP32 or FP64
//  k_record         the draw record of one generation (parity checks)
//  k_best           y* = min fitness per executor (Sec. III-B)
//  k_plain_*        plain path: one executor, one generation, three launches
//  k_fused_small    batched path, D <= 32: one CTA per executor, one thread per
//                   individual, population/trials/R resident in shared memory
//                   for all fused generations; the pbest pool is re-ranked
//                   each generation among the old pool and the improved
//  k_fused_general  batched path, any D: one CTA per executor, one warp per
//                   individual, population in global memory (L2-resident),
//                   R^T staged in shared memory when it fits
//  k_outer_*        the evolver of Alg. 3 (rand/1/bin, decode, selection)
#include <cstdio>

#include "block.cuh"
#include "internal.h"

namespace metade {

// ------------------------------------------------------------ problems
__global__ void k_pad_problems(const float* __restrict__ rot_in, const float* __restrict__ shift_in,
                               const long long* __restrict__ rot_in_off, const int* __restrict__ shift_in_off,
                               const int* __restrict__ dims, const long long* __restrict__ rot_off,
                               const int* __restrict__ shift_off, float* rot, float* rotT, float* shift) {
    const int p = blockIdx.x, r = blockIdx.y;
    const int dim = dims[p], dp = (dim + 3) & ~3;
    if (r >= dim) return;
    const float* Rin = rot_in + rot_in_off[p];
    for (int c = threadIdx.x; c < dp; c += blockDim.x) {
        rot[rot_off[p] + (long long)r * dp + c] = c < dim ? Rin[(long long)r * dim + c] : 0.0f;
        // rotT row r holds column r of R: rotT[r][c] = R[c][r]
        rotT[rot_off[p] + (long long)r * dp + c] = c < dim ? Rin[(long long)c * dim + r] : 0.0f;
    }
    if (r == 0)
        for (int j = threadIdx.x; j < dp; j += blockDim.x)
            shift[shift_off[p] + j] = j < dim ? shift_in[shift_in_off[p] + j] : 0.0f;
}

cudaError_t launch_pad_problems(const float* rot_in, const float* shift_in, const long long* rot_in_off,
                                const int* shift_in_off, const int* dims, const long long* rot_off,
                                const int* shift_off, int n_prob, int max_dim, float* rot, float* rotT,
                                float* shift, cudaStream_t st) {
    dim3 grid(n_prob, max_dim);
    k_pad_problems<<<grid, 128, 0, st>>>(rot_in, shift_in, rot_in_off, shift_in_off, dims, rot_off, shift_off,
                                         rot, rotT, shift);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- init
// Thread per (individual, 4-coordinate chunk): slot j/4 of generation
// 0xFFFFFFFF; x = lo + (hi - lo) U rounded once (fmaf).  Pad columns zero.
__global__ void k_init(const InstDesc* __restrict__ desc, float* pop, Key key, uint32_t epoch_arg,
                       const uint32_t* epoch_dev, float lo, float hi) {
    const InstDesc d = desc[blockIdx.y];
    const uint32_t epoch = epoch_dev ? *epoch_dev : epoch_arg;
    const int chunks = d.dpad >> 2;
    const float span = hi - lo;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.np * chunks; e += gridDim.x * blockDim.x) {
        const int i = e / chunks, q = e - i * chunks;
        const uint4 w = philox((uint32_t)d.stream, kInitGen, (uint32_t)i, (epoch << 16) | (uint32_t)q, key);
        float x[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) x[t] = (4 * q + t < d.dim) ? fmaf(span, uniform24(word_of(w, t)), lo) : 0.0f;
        *reinterpret_cast<float4*>(pop + d.pop_off + (long long)i * d.dpad + 4 * q) = make_float4(x[0], x[1], x[2], x[3]);
    }
}

cudaError_t launch_init(const InstDesc* desc, int n_inst, int max_np, int max_dpad, float* pop, Key key,
                        uint32_t epoch, const uint32_t* epoch_dev, float lo, float hi, cudaStream_t st) {
    if (n_inst <= 0) return cudaSuccess;
    const int work = max_np * (max_dpad / 4);
    dim3 grid((work + 255) / 256, n_inst);
    k_init<<<grid, 256, 0, st>>>(desc, pop, key, epoch, epoch_dev, lo, hi);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- eval
// Warp per row.  Dynamic shared: per warp 4 * max_dpad floats.  Population
// rows (pt_inst == nullptr): row r of the fitness layout, executor
// row_inst[r].  Caller-given points (pt_inst != nullptr): point r is
// pop[r * ldx ..], of executor pt_inst[r]; an executor id outside
// [0, n_inst) or a dimension above ldx latches EINVAL (1) in *status and
// yields NaN.
template <bool F64>
__global__ void __launch_bounds__(256) k_eval(const InstDesc* __restrict__ desc, const int* __restrict__ row_inst,
                                              long long n_rows, const float* __restrict__ pop,
                                              const float* __restrict__ rotT, const float* __restrict__ shift,
                                              void* f_out, int nan_inf, int scratch, int skip_tc,
                                              const float* __restrict__ mlp_x, const float* __restrict__ mlp_y,
                                              const int* __restrict__ pt_inst, int ldx, int n_inst, int* status) {
    extern __shared__ __align__(16) float sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* wb = sm + (size_t)warp * scratch;
    for (long long row = (long long)blockIdx.x * (blockDim.x >> 5) + warp; row < n_rows;
         row += (long long)gridDim.x * (blockDim.x >> 5)) {
        const int k = pt_inst ? pt_inst[row] : row_inst[row];
        if (pt_inst && (k < 0 || k >= n_inst || desc[k].dim > ldx)) {  // warp-uniform
            if (lane == 0) {
                set_status(status, 1);
                if (F64) reinterpret_cast<double*>(f_out)[row] = __longlong_as_double(0x7FF8000000000000LL);
                else reinterpret_cast<float*>(f_out)[row] = __int_as_float(0x7FC00000);
            }
            continue;
        }
        const InstDesc d = desc[k];
        if (skip_tc && (d.on_tc || d.obj == kMlp)) continue;  // warp-uniform: one row per warp
        const long long i = row - d.fit_off;
        const float* x = pt_inst ? pop + row * (long long)ldx : pop + d.pop_off + i * d.dpad;
        const float* o = shift + d.shift_off;
        const float* RT = rotT + d.rot_off;
        if (d.obj == kMlp) {  // warp-uniform; lanes take inputs n = lane, lane + 32, ...
            const int h = mlp_hidden(d.dim);
            if (F64) {  // teacher outputs recomputed in FP64 from the shift
                double s = 0.0;
                for (int n = lane; n < kMlpN; n += 32) {
                    double xv[kMlpIn], yt[kMlpOut], y[kMlpOut];
#pragma unroll
                    for (int q = 0; q < kMlpIn; ++q) xv[q] = (double)mlp_x[n * kMlpIn + q];
                    mlp_forward<double>(h, o, xv, yt);
                    mlp_forward<double>(h, x, xv, y);
                    s += (y[0] - yt[0]) * (y[0] - yt[0]) + (y[1] - yt[1]) * (y[1] - yt[1]);
                }
                const double f = warp_sum(s) / (kMlpN * kMlpOut);
                if (lane == 0) reinterpret_cast<double*>(f_out)[row] = nan_inf ? nan_to_inf(f) : f;
            } else {
                float s = 0.0f;
                for (int n = lane; n < kMlpN; n += 32) {
                    float xv[kMlpIn], y[kMlpOut];
#pragma unroll
                    for (int q = 0; q < kMlpIn; ++q) xv[q] = mlp_x[n * kMlpIn + q];
                    mlp_forward<float>(h, x, xv, y);
                    const float e0 = y[0] - mlp_y[d.aux + 2 * n], e1 = y[1] - mlp_y[d.aux + 2 * n + 1];
                    s += fmaf(e0, e0, e1 * e1);
                }
                const float f = warp_sum(s) * (1.0f / (kMlpN * kMlpOut));
                if (lane == 0) reinterpret_cast<float*>(f_out)[row] = nan_inf ? nan_to_inf(f) : f;
            }
            continue;
        }
        if (F64) {
            double* db = reinterpret_cast<double*>(wb);
            const double f = warp_eval64(d.obj, d.dim, x, o, RT, d.dpad, db, db + d.dpad);
            if (lane == 0) reinterpret_cast<double*>(f_out)[row] = nan_inf ? nan_to_inf(f) : f;
        } else {
            float* db = wb;
            float* zb = wb + d.dpad;
            for (int j = lane; j < d.dpad; j += 32) db[j] = j < d.dim ? x[j] - o[j] : 0.0f;
            __syncwarp();
            warp_rotate<float>(d.dim, RT, d.dpad, db, zb);
            __syncwarp();
            const float f = warp_objective<float>(d.obj, d.dim, zb);
            if (lane == 0) reinterpret_cast<float*>(f_out)[row] = nan_inf ? nan_to_inf(f) : f;
            __syncwarp();
        }
    }
}

static int g_num_sms = 0;
static int num_sms() {
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 132;
    }
    return g_num_sms;
}

cudaError_t launch_eval(const InstDesc* desc, const int* row_inst, long long n_rows, const float* pop,
                        const float* rotT, const float* shift, bool f64, void* f_out, bool nan_inf, int max_dpad,
                        cudaStream_t st, bool skip_tc, const float* mlp_x, const float* mlp_y, const int* pt_inst,
                        int ldx, int n_inst, int* status) {
    if (n_rows <= 0) return cudaSuccess;
    const int scratch = 4 * max_dpad;  // floats per warp: two buffers of max_dpad doubles
    const size_t smem = (size_t)8 * scratch * sizeof(float);
    long long blocks = (n_rows + 7) / 8;
    const long long cap = (long long)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    if (f64) {
        cudaFuncSetAttribute(k_eval<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_eval<true><<<(unsigned)blocks, 256, smem, st>>>(desc, row_inst, n_rows, pop, rotT, shift, f_out,
                                                          nan_inf, scratch, skip_tc ? 1 : 0, mlp_x, mlp_y,
                                                          pt_inst, ldx, n_inst, status);
    } else {
        cudaFuncSetAttribute(k_eval<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_eval<false><<<(unsigned)blocks, 256, smem, st>>>(desc, row_inst, n_rows, pop, rotT, shift, f_out,
                                                           nan_inf, scratch, skip_tc ? 1 : 0, mlp_x, mlp_y,
                                                           pt_inst, ldx, n_inst, status);
    }
    return cudaGetLastError();
}

// -------------------------------------------------------------- record
// Block per executor, thread per individual; the pool and best come from the
// generation-start fitness.  Dynamic shared: topk [np] + 64 words.
__global__ void k_record(StepArgs a, int* rec) {
    extern __shared__ int smi[];
    const int k = blockIdx.x;
    const InstDesc d = a.desc[k];
    const float* f = a.fit + d.fit_off;
    int* topk = smi;
    const Strat s = load_strat(a.theta + 6 * k, d.np);
    if (!s.ok) {
        if (threadIdx.x == 0) set_status(a.status, 1);
        return;
    }
    block_topk(f, d.np, d.kp, topk);
    __syncthreads();
    const int best = topk[0];
    for (int i = threadIdx.x; i < d.np; i += blockDim.x) {
        const Ctr c = make_ctr(a.key, (uint32_t)d.stream, a.gen0, (uint32_t)i, a.epoch_dev ? *a.epoch_dev : a.epoch);
        Indiv v;
        indiv_setup(s, c, i, d.np, d.dim, d.kp, topk, best, v);
        int* q = rec + (long long)(d.fit_off + i) * kRecFields;
        q[0] = v.ibl;
        q[1] = v.ibr;
        q[2] = v.jrand;
        q[3] = v.nstart;
        q[4] = s.cs == 2 ? exp_length(c, d.dim, s.cri) : 0;
        q[5] = (int)v.kraw;
        q[6] = v.pbest;
        q[7] = best;
        q[8] = s.m;
#pragma unroll
        for (int t = 0; t < 9; ++t) q[9 + t] = v.r[t];
    }
}

cudaError_t launch_record(const StepArgs& a, int n_inst, int max_np, int* rec, cudaStream_t st) {
    k_record<<<n_inst, 256, (size_t)max_np * sizeof(int), st>>>(a, rec);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- best
__global__ void k_best(const InstDesc* __restrict__ desc, const float* __restrict__ fit, float* best_f,
                       int* best_i) {
    __shared__ int red[64];
    const InstDesc d = desc[blockIdx.x];
    const int b = block_argmin(fit + d.fit_off, d.np, red);
    if (threadIdx.x == 0) {
        if (best_f) best_f[blockIdx.x] = fit[d.fit_off + b];
        if (best_i) best_i[blockIdx.x] = b;
    }
}

cudaError_t launch_best(const InstDesc* desc, int n_inst, const float* fit, float* best_f, int* best_i,
                        cudaStream_t st) {
    if (n_inst <= 0) return cudaSuccess;
    k_best<<<n_inst, 256, 0, st>>>(desc, fit, best_f, best_i);
    return cudaGetLastError();
}

// ---------------------------------------------------------- plain path
// The FP32 baseline: one executor per launch, one generation per launch,
// everything through global memory, no fusion, no graph, no tuning.  The
// launch is cooperative (all its CTAs resident at once), so the generation's
// three phases -- pbest pool, trials with their evaluation, selection -- are
// separated by grid-wide barriers inside the one launch: every trial is built
// from the generation-start population before any row is replaced.

// Polls of the grid barrier before it gives up: with a 100 ns back-off per
// poll, well over 0.1 s, far beyond any phase of one plain generation.
constexpr uint32_t kGridWaitLimit = 1u << 21;

// Grid-wide barrier of a cooperative launch.  Thread 0 of every CTA arrives
// by one atomic increment of *count (after a fence, so the CTA's writes are
// visible first) and polls until *count reaches `target`: the arrivals of
// this barrier and of the call's earlier ones.  Gives up after
// kGridWaitLimit polls, latching METADE_ETIMEOUT (4), and the CTA returns.
__device__ bool grid_barrier(unsigned* count, unsigned target, int* status) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        bool ok = false;
        for (uint32_t it = 0; it < kGridWaitLimit; ++it) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if (v >= target) {
                ok = true;
                break;
            }
            __nanosleep(100);
        }
        if (!ok) set_status(status, 4);
        __threadfence();
        ok_s = ok ? 1 : 0;
    }
    __syncthreads();
    return ok_s != 0;
}

// Grid: ceil(NP / 8) CTAs of 256 threads (a warp per individual).  Dynamic
// shared memory: 4 dpad floats per warp.  bar counts barrier arrivals within
// the caller's sequence of launches; this launch's barriers wait for
// base + gridDim.x and base + 2 gridDim.x.
__global__ void __launch_bounds__(256) k_plain_gen(StepArgs a, int k, int* topk, float* uscr, float* fuscr,
                                                   unsigned* bar, unsigned base) {
    extern __shared__ __align__(16) float sm[];
    const InstDesc d = a.desc[k];
    const Strat s = load_strat(a.theta + 6 * k, d.np);
    // An invalid theta (the same decision in every CTA), or a barrier of an
    // earlier launch that gave up: no work, but every CTA still counts its two
    // arrivals so that the barriers of later launches keep their targets.
    const bool skip = !s.ok || *(volatile int*)a.status == 4;
    if (skip) {
        if (threadIdx.x == 0) atomicAdd(bar, 2u);
        if (!s.ok && blockIdx.x == 0 && threadIdx.x == 0) set_status(a.status, 1);
        return;
    }
    // phase 1: best and the pbest pool from the generation-start fitness
    if (blockIdx.x == 0) block_topk_staged(a.fit + d.fit_off, d.np, d.kp, topk);
    if (!grid_barrier(bar, base + gridDim.x, a.status)) return;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + warp;
    const float* o = a.shift + d.shift_off;
    const float* RT = a.rotT + d.rot_off;
    // phase 2: trial and its FP32 evaluation, a warp per individual
    if (i < d.np) {
        float* db = sm + (size_t)warp * 4 * d.dpad;
        float* zb = db + d.dpad;
        const Ctr c = make_ctr(a.key, (uint32_t)d.stream, a.gen0, (uint32_t)i, a.epoch_dev ? *a.epoch_dev : a.epoch);
        Indiv v;
        indiv_setup(s, c, i, d.np, d.dim, d.kp, topk, topk[0], v);
        const int L = s.cs == 2 ? exp_length(c, d.dim, s.cri) : 0;
        warp_trial(s, c, v, i, d.dim, L, a.pop + d.pop_off, d.dpad, o, a.lo, a.hi,
                   uscr + d.pop_off + (long long)i * d.dpad, db);
        __syncwarp();
        warp_rotate<float>(d.dim, RT, d.dpad, db, zb);
        __syncwarp();
        const float f = warp_objective<float>(d.obj, d.dim, zb);
        if (lane == 0) fuscr[d.fit_off + i] = nan_to_inf(f);
        __syncwarp();
    }
    if (!grid_barrier(bar, base + 2 * gridDim.x, a.status)) return;

    // phase 3: greedy selection (near ties decided precisely) and row copy
    if (i >= d.np) return;
    float* X = a.pop + d.pop_off + (long long)i * d.dpad;
    const float* U = uscr + d.pop_off + (long long)i * d.dpad;
    float fn = fuscr[d.fit_off + i];
    const float fx = a.fit[d.fit_off + i];
    bool take;
    bool tie = near_tie(fn, fx, tie_band(d.dim));
    if (tie) {
        bool diff = false;
        for (int j = lane; j < d.dim; j += 32) diff = diff || (U[j] != X[j]);
        if (!__any_sync(kFull, diff)) tie = false, fn = fx;  // trial == target
    }
    if (tie && a.tie_fp64) {
        double* db = reinterpret_cast<double*>(sm + (size_t)warp * 4 * d.dpad);
        const double eu = nan_to_inf(warp_eval64(d.obj, d.dim, U, o, RT, d.dpad, db, db + d.dpad));
        const double ex = nan_to_inf(warp_eval64(d.obj, d.dim, X, o, RT, d.dpad, db, db + d.dpad));
        take = eu <= ex;
        if (take) fn = fminf((float)eu, fx);
    } else if (tie) {
        float* zb = sm + (size_t)warp * 4 * d.dpad;
        warp_rotate_pair(d.dim, RT, d.dpad, X, U, o, zb, zb + d.dpad);
        __syncwarp();
        const float df = warp_diff(d.obj, d.dim, zb, zb + d.dpad);
        take = df <= 0.0f;
        if (take) fn = fx + df;
    } else {
        take = fn <= fx;
    }
    if (take) {
        for (int j = lane * 4; j < d.dpad; j += 128)
            *reinterpret_cast<float4*>(X + j) = *reinterpret_cast<const float4*>(U + j);
        if (lane == 0) a.fit[d.fit_off + i] = fn;
    }
}

cudaError_t launch_plain_generation(const StepArgs& a, int k, const InstDesc& d, float* uscr, float* fuscr,
                                    int* topk, unsigned* bar, unsigned base, cudaStream_t st) {
    const int blocks = (d.np + 7) / 8;
    const size_t smem = (size_t)8 * 4 * d.dpad * sizeof(float);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_plain_gen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    StepArgs aa = a;
    int kk = k;
    void* args[] = {&aa, &kk, &topk, &uscr, &fuscr, &bar, &base};
    return cudaLaunchCooperativeKernel((const void*)k_plain_gen, dim3(blocks), dim3(256), args, smem, st);
}

// ------------------------------------------------ batched path, small D
// Thread-level trial: individual i's trial row into U (shared, stride ds) and
// u - o into registers.
template <int DMAX>
__device__ __forceinline__ void thread_trial(const Strat& s, const Ctr& c, const Indiv& v, int i, int dim, int ds,
                                             int L, const float* X, const float* o, float lo, float hi, float* U,
                                             float (&dreg)[DMAX]) {
    const float F = s.F, K = (float)v.kraw * (1.0f / 16777216.0f);
    const float* xl = X + v.ibl * ds;
    const float* xr = X + v.ibr * ds;
    const float* xi = X + i * ds;
    const bool dir = s.bl != s.br;
#pragma unroll
    for (int j4 = 0; j4 < DMAX; j4 += 4) {
        if (j4 < dim) {
            const float4 a = *reinterpret_cast<const float4*>(xl + j4);
            const float4 b = *reinterpret_cast<const float4*>(xr + j4);
            const float4 x = *reinterpret_cast<const float4*>(xi + j4);
            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int q = 0; q < s.dn; ++q) {
                const float4 p = *reinterpret_cast<const float4*>(X + diff_plus(v, s.a, q) * ds + j4);
                const float4 m = *reinterpret_cast<const float4*>(X + diff_minus(v, s.a, q) * ds + j4);
                sum.x += p.x - m.x; sum.y += p.y - m.y; sum.z += p.z - m.z; sum.w += p.w - m.w;
            }
            const uint4 w = (s.cs == 1) ? c.slot(4 + (uint32_t)(j4 >> 2)) : make_uint4(0, 0, 0, 0);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
            const float xv[4] = {x.x, x.y, x.z, x.w}, sv[4] = {sum.x, sum.y, sum.z, sum.w};
            float uo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = j4 + q;
                float vj = av[q];
                if (dir) vj += F * (bv[q] - av[q]);
                vj += F * sv[q];
                float u;
                if (s.cs == 3) {
                    u = xv[q] + K * (vj - xv[q]);
                } else {
                    bool take;
                    if (s.cs == 1) {
                        take = ((word_of(w, q) >> 8) < s.cri) || (j == v.jrand);
                    } else {
                        int off = j - v.nstart;
                        if (off < 0) off += dim;
                        take = off < L;
                    }
                    u = take ? vj : xv[q];
                }
                u = fminf(fmaxf(u, lo), hi);
                if (j >= dim) u = 0.0f;
                uo[q] = u;
                dreg[j] = (j < dim) ? (u - o[j]) : 0.0f;
            }
            *reinterpret_cast<float4*>(U + i * ds + j4) = make_float4(uo[0], uo[1], uo[2], uo[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) dreg[j4 + q] = 0.0f;
        }
    }
}

// f(u) - f(x) for one individual by its own thread (selection ties): x - o
// and u - x are formed once in registers, then both rotations share R loads.
// Out of line: inlined, its code (both rotations and every objective's
// difference form) spreads the fused loop over more instruction cache lines
// (measured 3.5% slower).
template <int DMAX>
__device__ __noinline__ float diff_small(int obj, int dim, const float* u, const float* x, const float* o,
                                         const float* R) {
    float dx[DMAX], dl[DMAX];
#pragma unroll
    for (int c4 = 0; c4 < DMAX / 4; ++c4) {  // whole chunks below dim; padding columns are zero
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (4 * c4 < dim) {
            const float4 xv = reinterpret_cast<const float4*>(x)[c4], uv = reinterpret_cast<const float4*>(u)[c4];
            const float4 ov = reinterpret_cast<const float4*>(o)[c4];
            a = make_float4(xv.x - ov.x, xv.y - ov.y, xv.z - ov.z, xv.w - ov.w);
            b = make_float4(uv.x - xv.x, uv.y - xv.y, uv.z - xv.z, uv.w - xv.w);
        }
        dx[4 * c4] = a.x; dx[4 * c4 + 1] = a.y; dx[4 * c4 + 2] = a.z; dx[4 * c4 + 3] = a.w;
        dl[4 * c4] = b.x; dl[4 * c4 + 1] = b.y; dl[4 * c4 + 2] = b.z; dl[4 * c4 + 3] = b.w;
    }
    DiffAcc acc;
    diff_init(acc);
    for (int r = 0; r < dim; ++r) {
        const float4* Rr = reinterpret_cast<const float4*>(R + r * DMAX);
        float z = 0.f, dz = 0.f;
#pragma unroll
        for (int c4 = 0; c4 < DMAX / 4; ++c4) {
            const float4 q = Rr[c4];
            z = fmaf(q.x, dx[4 * c4], z);
            z = fmaf(q.y, dx[4 * c4 + 1], z);
            z = fmaf(q.z, dx[4 * c4 + 2], z);
            z = fmaf(q.w, dx[4 * c4 + 3], z);
            dz = fmaf(q.x, dl[4 * c4], dz);
            dz = fmaf(q.y, dl[4 * c4 + 1], dz);
            dz = fmaf(q.z, dl[4 * c4 + 2], dz);
            dz = fmaf(q.w, dl[4 * c4 + 3], dz);
        }
        diff_push(obj, acc, z, dz);
    }
    return diff_finish(obj, acc, dim);
}

// FP64 re-evaluation of a near tie by one thread, kept out of line: it is
// rare, and inlined it would spread the fused loop's code.  Returns the
// decision and, when taken, the stored value min(f32(f64 f(u)), f(x)) in fn.
__device__ __noinline__ bool tie_fp64_small(int obj, int dim, int dmax, const float* u, const float* x,
                                            const float* o, const float* R, float fx, float& fn) {
    const double eu = nan_to_inf(eval64_seq(obj, dim, dmax, u, o, R));
    const double ex = nan_to_inf(eval64_seq(obj, dim, dmax, x, o, R));
    if (eu <= ex) fn = fminf((float)eu, fx);
    return eu <= ex;
}

// f(u) of one individual from z = R (u - o), rows four at a time, the
// objective a template parameter: one objective dispatch per individual
// rather than one per four rows (1% faster on the small-D kernel).
template <int DMAX, int OBJ>
__device__ __forceinline__ float small_eval(int dim, const float* R, const float (&dreg)[DMAX], const float* isq) {
    ObjR acc;
    int r = 0;
    for (; r + 4 <= dim; r += 4) {
        const float4* R0 = reinterpret_cast<const float4*>(R + (r + 0) * DMAX);
        const float4* R1 = reinterpret_cast<const float4*>(R + (r + 1) * DMAX);
        const float4* R2 = reinterpret_cast<const float4*>(R + (r + 2) * DMAX);
        const float4* R3 = reinterpret_cast<const float4*>(R + (r + 3) * DMAX);
        float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
        for (int c4 = 0; c4 < DMAX / 4; ++c4) {
            const float d0 = dreg[4 * c4], d1 = dreg[4 * c4 + 1], d2 = dreg[4 * c4 + 2], d3 = dreg[4 * c4 + 3];
            const float4 q0 = R0[c4], q1 = R1[c4], q2 = R2[c4], q3 = R3[c4];
            z0 = fmaf(q0.x, d0, z0); z0 = fmaf(q0.y, d1, z0); z0 = fmaf(q0.z, d2, z0); z0 = fmaf(q0.w, d3, z0);
            z1 = fmaf(q1.x, d0, z1); z1 = fmaf(q1.y, d1, z1); z1 = fmaf(q1.z, d2, z1); z1 = fmaf(q1.w, d3, z1);
            z2 = fmaf(q2.x, d0, z2); z2 = fmaf(q2.y, d1, z2); z2 = fmaf(q2.z, d2, z2); z2 = fmaf(q2.w, d3, z2);
            z3 = fmaf(q3.x, d0, z3); z3 = fmaf(q3.y, d1, z3); z3 = fmaf(q3.z, d2, z3); z3 = fmaf(q3.w, d3, z3);
        }
        acc.push4_t<OBJ>(z0, z1, z2, z3, isq + r);
    }
    for (; r < dim; ++r) {
        const float4* Rr = reinterpret_cast<const float4*>(R + r * DMAX);
        float z = 0.0f;
#pragma unroll
        for (int c4 = 0; c4 < DMAX / 4; ++c4) {
            const float4 rr = Rr[c4];
            z = fmaf(rr.x, dreg[4 * c4 + 0], z);
            z = fmaf(rr.y, dreg[4 * c4 + 1], z);
            z = fmaf(rr.z, dreg[4 * c4 + 2], z);
            z = fmaf(rr.w, dreg[4 * c4 + 3], z);
        }
        acc.push_t<OBJ>(z, isq[r]);
    }
    return acc.finish(OBJ, dim);
}

__host__ __device__ inline int small_stride(int dpad) { return ((dpad >> 2) & 1) ? dpad : dpad + 4; }

// One executor, all fused generations, everything resident in shared memory;
// the objective is a template parameter so the hot loop has no objective branch.
template <int DMAX>
__device__ __forceinline__ void small_executor(const StepArgs& a, int k, const InstDesc& d, const Strat& s,
                                               float* sm) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int np = d.np, dim = d.dim, dp = d.dpad, ds = small_stride(dp);
    const float band = tie_band(dim);
    float* X = sm;
    float* U = X + np * ds;
    float* R = U + np * ds;
    float* o = R + dim * DMAX;
    float* isq = o + DMAX;
    float* f = isq + DMAX;
    float* fu = f + np;
    int* topk = reinterpret_cast<int*>(fu + np);
    int* red = topk + np;
    // pbest pool bookkeeping: the candidates for the next generation's pool
    // (listed by the selection), their fitness, pool membership, the count
    int* cand = red + 64;
    float* candf = reinterpret_cast<float*>(cand + np);
    int* inpool = reinterpret_cast<int*>(candf + np);
    int* ncand = inpool + np;
    const uint32_t epoch = a.epoch_dev ? *a.epoch_dev : a.epoch;
    float* gpop = a.pop + d.pop_off;
    const int chunks = dp >> 2;
    for (int e = tid; e < np * chunks; e += nt) {
        const int i = e / chunks, q = e - i * chunks;
        *reinterpret_cast<float4*>(X + i * ds + 4 * q) =
            *reinterpret_cast<const float4*>(gpop + (long long)i * dp + 4 * q);
    }
    const float* gR = a.rot + d.rot_off;
    for (int e = tid; e < dim * DMAX; e += nt) {
        const int r = e / DMAX, cc = e - r * DMAX;
        R[e] = cc < dp ? gR[(long long)r * dp + cc] : 0.0f;
    }
    for (int j = tid; j < DMAX; j += nt) {
        o[j] = j < dp ? a.shift[d.shift_off + j] : 0.0f;
        isq[j] = (float)(0.15915494309189535 / sqrt((double)(j + 1)));  // Griewank's 1/(2 pi sqrt j)
    }
    for (int i = tid; i < np; i += nt) {
        f[i] = a.fit[d.fit_off + i];
        inpool[i] = 0;
    }
    if (tid == 0) *ncand = 0;
    __syncthreads();
    const bool pb = s.uses_pbest();
    for (int g = 0; g < a.n_gens; ++g) {
        const uint32_t gen = a.gen0 + (uint32_t)g;
        int best;
        if (pb) {
            if (g == 0) {
                block_topk(f, np, d.kp, topk);
                __syncthreads();
                for (int t = tid; t < d.kp; t += nt) inpool[topk[t]] = 1;
            } else {
                // Stored fitness never rises (greedy selection), so an individual
                // outside the old pool whose fitness did not fall still has k_p
                // better ones: the new pool lies within the old pool and the
                // individuals whose fitness fell.  Everyone better than a pool
                // member is in the pool, so its rank among these candidates is
                // its exact rank by (f, index); a non-member ranks >= k_p there.
                const int m = *ncand;
                for (int t = tid; t < m; t += nt) {
                    const int ci = cand[t];
                    const float fc = candf[t];
                    int rank = 0;
                    for (int j = 0; j < m; ++j) rank += better(candf[j], cand[j], fc, ci) ? 1 : 0;
                    inpool[ci] = rank < d.kp;
                    if (rank < d.kp) topk[rank] = ci;
                }
                __syncthreads();
                if (tid == 0) *ncand = 0;
            }
            best = topk[0];
        } else {
            best = block_argmin(f, np, red);
        }
        for (int i = tid; i < np; i += nt) {
            const Ctr c = make_ctr(a.key, (uint32_t)d.stream, gen, (uint32_t)i, epoch);
            Indiv v;
            indiv_setup(s, c, i, np, dim, d.kp, pb ? topk : nullptr, best, v);
            const int L = s.cs == 2 ? exp_length(c, dim, s.cri) : 0;
            float dreg[DMAX];
            thread_trial<DMAX>(s, c, v, i, dim, ds, L, X, o, a.lo, a.hi, U, dreg);
            float fv;
            switch (d.obj) {
            case kSphere: fv = small_eval<DMAX, kSphere>(dim, R, dreg, isq); break;
            case kRosenbrock: fv = small_eval<DMAX, kRosenbrock>(dim, R, dreg, isq); break;
            case kRastrigin: fv = small_eval<DMAX, kRastrigin>(dim, R, dreg, isq); break;
            case kGriewank: fv = small_eval<DMAX, kGriewank>(dim, R, dreg, isq); break;
            case kAckley: fv = small_eval<DMAX, kAckley>(dim, R, dreg, isq); break;
            default: fv = small_eval<DMAX, kSchwefel12>(dim, R, dreg, isq); break;
            }
            fu[i] = nan_to_inf(fv);
        }
        __syncthreads();
        for (int i = tid; i < np; i += nt) {
            float fn = fu[i];
            const float fx = f[i];
            bool take;
            bool same = near_tie(fn, fx, band);
            if (same) {  // padding columns are zero in both rows
                const float4* u4 = reinterpret_cast<const float4*>(U + i * ds);
                const float4* x4 = reinterpret_cast<const float4*>(X + i * ds);
                for (int q = 0; q < chunks && same; ++q) {
                    const float4 p = u4[q], r = x4[q];
                    same = p.x == r.x && p.y == r.y && p.z == r.z && p.w == r.w;
                }
            }
            if (same) {
                take = true;  // the trial is the target: nothing changes
                fn = fx;
            } else if (near_tie(fn, fx, band)) {
                if (a.tie_fp64) {
                    take = tie_fp64_small(d.obj, dim, DMAX, U + i * ds, X + i * ds, o, R, fx, fn);
                } else {
                    const float df = diff_small<DMAX>(d.obj, dim, U + i * ds, X + i * ds, o, R);
                    take = df <= 0.0f;
                    if (take) fn = fx + df;
                }
            } else {
                take = fn <= fx;
            }
            if (pb && (inpool[i] || (take && fn < fx))) {  // candidate for the next pool
                const int slot = atomicAdd(ncand, 1);
                cand[slot] = i;
                candf[slot] = take ? fn : fx;
            }
            if (take) {
                for (int q = 0; q < chunks; ++q)
                    *reinterpret_cast<float4*>(X + i * ds + 4 * q) =
                        *reinterpret_cast<const float4*>(U + i * ds + 4 * q);
                f[i] = fn;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < np * chunks; e += nt) {
        const int i = e / chunks, q = e - i * chunks;
        *reinterpret_cast<float4*>(gpop + (long long)i * dp + 4 * q) =
            *reinterpret_cast<const float4*>(X + i * ds + 4 * q);
    }
    for (int i = tid; i < np; i += nt) a.fit[d.fit_off + i] = f[i];
    const int b = block_argmin(f, np, red);
    if (tid == 0 && a.best_f) a.best_f[k] = f[b];
    if (tid == 0 && a.best_i) a.best_i[k] = b;
    __syncthreads();
}

template <int DMAX>
__global__ void __launch_bounds__(256, 2) k_fused_small(StepArgs a, const int* __restrict__ work, int n_work) {
    extern __shared__ __align__(16) float sm[];
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const int k = work[w];
        const InstDesc d = a.desc[k];
        const Strat s = load_strat(a.theta + 6 * k, d.np);
        if (!s.ok) {
            if (threadIdx.x == 0) set_status(a.status, 1);
            continue;
        }
        small_executor<DMAX>(a, k, d, s, sm);
    }
}

int small_dmax_for(int dim) {
    if (dim <= 4) return 4;
    if (dim <= 8) return 8;
    if (dim <= 12) return 12;
    if (dim <= 16) return 16;
    if (dim <= 20) return 20;
    if (dim <= 24) return 24;
    if (dim <= 32) return 32;
    return 0;
}

size_t fused_smem_small(int dmax, int max_np) {
    const int ds = small_stride(dmax);
    return sizeof(float) * ((size_t)2 * max_np * ds + (size_t)dmax * dmax + 2 * dmax + 2 * (size_t)max_np) +
           sizeof(int) * ((size_t)4 * max_np + 64 + 1);
}

// ---------------------------------------------- batched path, general D
// Shared layout: f[np], fu[np], topk[np], red[64], R^T [dim][dpad] (optional),
// then per warp 4 * max_dpad floats (float trial buffers or double tie buffers).
__global__ void __launch_bounds__(512) k_fused_general(StepArgs a, const int* __restrict__ work, int n_work,
                                                       float* uscr, int rot_smem, int max_np, int max_dpad) {
    extern __shared__ __align__(16) float sm[];
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    float* f = sm;
    float* fu = f + max_np;
    int* topk = reinterpret_cast<int*>(fu + max_np);
    int* red = topk + max_np;
    float* rs = sm + ((3 * max_np + 64 + 3) & ~3);
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const int k = work[w];
        const InstDesc d = a.desc[k];
        const int np = d.np, dim = d.dim, dp = d.dpad;
        const float band = tie_band(dim);
        float* RTs = rs;
        float* wb = rs + (rot_smem ? (size_t)max_dpad * max_dpad : 0) + (size_t)warp * 4 * max_dpad;
        float* db = wb;
        float* zb = wb + max_dpad;
        const Strat s = load_strat(a.theta + 6 * k, np);
        if (!s.ok) {
            if (tid == 0) set_status(a.status, 1);
            continue;
        }
        const uint32_t epoch = a.epoch_dev ? *a.epoch_dev : a.epoch;
        float* X = a.pop + d.pop_off;
        float* Ug = uscr + d.pop_off;
        const float* o = a.shift + d.shift_off;
        const float* RT = a.rotT + d.rot_off;
        if (rot_smem) {
            for (int e = tid; e < dim * (dp >> 2); e += nt)
                reinterpret_cast<float4*>(RTs)[e] = reinterpret_cast<const float4*>(RT)[e];
            RT = RTs;
        }
        for (int i = tid; i < np; i += nt) f[i] = a.fit[d.fit_off + i];
        __syncthreads();
        const bool pb = s.uses_pbest();
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
            for (int i = warp; i < np; i += nw) {
                const Ctr c = make_ctr(a.key, (uint32_t)d.stream, gen, (uint32_t)i, epoch);
                Indiv v;
                indiv_setup(s, c, i, np, dim, d.kp, pb ? topk : nullptr, best, v);
                const int L = s.cs == 2 ? warp_exp_length(c, dim, s.cri) : 0;  // uniform over the warp
                warp_trial(s, c, v, i, dim, L, X, dp, o, a.lo, a.hi, Ug + (long long)i * dp, db);
                __syncwarp();
                warp_rotate<float>(dim, RT, dp, db, zb);
                __syncwarp();
                const float fv = warp_objective<float>(d.obj, dim, zb);
                if (lane == 0) fu[i] = nan_to_inf(fv);
                __syncwarp();
            }
            __syncthreads();
            for (int i = warp; i < np; i += nw) {
                float fn = fu[i];
                const float fx = f[i];
                float* Xi = X + (long long)i * dp;
                const float* Ui = Ug + (long long)i * dp;
                bool take;
                bool tie = near_tie(fn, fx, band);
                if (tie) {
                    bool diff = false;
                    for (int j = lane; j < dim; j += 32) diff = diff || (Ui[j] != Xi[j]);
                    if (!__any_sync(kFull, diff)) tie = false, fn = fx;  // trial == target
                }
                if (tie && a.tie_fp64) {
                    double* dd = reinterpret_cast<double*>(wb);
                    const double eu = nan_to_inf(warp_eval64(d.obj, dim, Ui, o, RT, dp, dd, dd + max_dpad));
                    const double ex = nan_to_inf(warp_eval64(d.obj, dim, Xi, o, RT, dp, dd, dd + max_dpad));
                    take = eu <= ex;
                    if (take) fn = fminf((float)eu, fx);
                } else if (tie) {
                    warp_rotate_pair_staged(dim, RT, dp, Xi, Ui, o, wb, max_dpad);
                    const float df = warp_diff(d.obj, dim, wb + 2 * max_dpad, wb + 3 * max_dpad);
                    __syncwarp();
                    take = df <= 0.0f;
                    if (take) fn = fx + df;
                } else {
                    take = fn <= fx;
                }
                if (take) {
                    for (int j = lane * 4; j < dp; j += 128)
                        *reinterpret_cast<float4*>(Xi + j) = *reinterpret_cast<const float4*>(Ui + j);
                    if (lane == 0) f[i] = fn;
                }
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

size_t fused_smem_general(int max_np, int max_dpad, int threads, bool rot_in_smem) {
    size_t words = 3 * (size_t)max_np + 64;
    words = (words + 3) & ~(size_t)3;
    if (rot_in_smem) words += (size_t)max_dpad * max_dpad;
    words += (size_t)(threads / 32) * 4 * max_dpad;
    return words * sizeof(float);
}

template <int DMAX>
static cudaError_t launch_small(const StepArgs& a, const int* work, int n_work, const FusedPlan& p, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_small<DMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    k_fused_small<DMAX><<<p.grid, p.threads, p.smem, st>>>(a, work, n_work);
    return cudaGetLastError();
}

cudaError_t launch_fused(const StepArgs& a, const int* work, int n_work, const FusedPlan& p, float* uscr,
                         cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    if (p.kind == 0) {
        switch (p.dmax) {
        case 4: return launch_small<4>(a, work, n_work, p, st);
        case 8: return launch_small<8>(a, work, n_work, p, st);
        case 12: return launch_small<12>(a, work, n_work, p, st);
        case 16: return launch_small<16>(a, work, n_work, p, st);
        case 20: return launch_small<20>(a, work, n_work, p, st);
        case 24: return launch_small<24>(a, work, n_work, p, st);
        case 32: return launch_small<32>(a, work, n_work, p, st);
        default: return cudaErrorInvalidValue;
        }
    }
    if (p.kind == 3) return launch_fused_tile(a, work, n_work, p, uscr, st);
    cudaError_t e = cudaFuncSetAttribute(k_fused_general, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    k_fused_general<<<p.grid, p.threads, p.smem, st>>>(a, work, n_work, uscr, p.rot_smem, p.max_np, p.max_dpad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- evolver
__constant__ float c_lb[6] = {0.f, 0.f, 1.f, 1.f, 1.f, 1.f};
__constant__ float c_ub[6] = {1.f, 1.f, 5.f, 5.f, 5.f, 4.f};

__global__ void k_outer_init(int n_total, int n_out, Key key, float* opop, float* ofit) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_total) return;
    const int g = e / n_out, i = e - g * n_out;
    const uint4 w0 = philox((uint32_t)g, kInitGen, (uint32_t)i, 0u, key);
    const uint4 w1 = philox((uint32_t)g, kInitGen, (uint32_t)i, 1u, key);
    const uint32_t ws[6] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y};
#pragma unroll
    for (int j = 0; j < 6; ++j) opop[(long long)e * 6 + j] = fmaf(c_ub[j] - c_lb[j], uniform24(ws[j]), c_lb[j]);
    ofit[e] = INFINITY;
}

// rand/1/bin with F = 0.5, CR = 0.9, then the floor decoding of Alg. 3.
__global__ void k_outer_trial(int n_total, int n_out, Key key, const uint32_t* gen_dev, uint32_t gen_arg,
                              const float* __restrict__ opop, float* trial, float* theta) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_total) return;
    const uint32_t gen = gen_dev ? *gen_dev : gen_arg;
    const int g = e / n_out, i = e - g * n_out;
    const float* P = opop + (long long)g * n_out * 6;
    const Ctr c = make_ctr(key, (uint32_t)g, gen, (uint32_t)i, 0u);
    const uint4 w0 = c.slot(0), w1 = c.slot(1), w2 = c.slot(2), w3 = c.slot(3);
    const int jrand = (int)below(w0.x, 6u);
    uint32_t w[12] = {w1.x, w1.y, w1.z, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    int r[9];
    distinct_draws(n_out, i, 3, w, r);
    const uint32_t xw[6] = {w2.x, w2.y, w2.z, w2.w, w3.x, w3.y};
    const uint32_t cri = threshold24(0.9f);
    float u[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const float v = P[r[0] * 6 + j] + 0.5f * (P[r[1] * 6 + j] - P[r[2] * 6 + j]);
        const bool take = ((xw[j] >> 8) < cri) || (j == jrand);
        float x = take ? v : P[i * 6 + j];
        x = fminf(fmaxf(x, c_lb[j]), c_ub[j]);
        u[j] = x;
        trial[(long long)e * 6 + j] = x;
    }
    float* th = theta + (long long)e * 6;
    th[0] = u[0];
    th[1] = u[1];
    const float top[4] = {4.f, 4.f, 4.f, 3.f};
#pragma unroll
    for (int j = 2; j < 6; ++j) th[j] = fminf(fmaxf(floorf(u[j]), 1.0f), top[j - 2]);
}

// PSO evolver (the supplement's comparison of evolvers; w = 0.729, c1 = c2 =
// 1.49).  opop / ofit hold the personal bests and their fitness; trial holds
// [position 6 | velocity 6] per particle.  Generation 0 evaluates the initial
// swarm (x = pbest, v = 0); later generations move every particle:
//   v <- w v + c1 r1 (pbest - x) + c2 r2 (gbest - x),  x <- clip(x + v)
// with gbest the run's personal best of lowest fitness (ties to the lower
// index) and r1 / r2 the uniforms of draw words 0..5 / 6..11 (slot = word / 4).
// The position is decoded into theta like a DE trial.
__global__ void k_pso_move(int n_total, int n_out, Key key, const uint32_t* gen_dev, uint32_t gen_arg,
                           const float* __restrict__ opop, const float* __restrict__ ofit, float* trial,
                           float* theta) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_total) return;
    const uint32_t gen = gen_dev ? *gen_dev : gen_arg;
    const int g = e / n_out, i = e - g * n_out;
    float* xv = trial + (long long)e * 12;
    const float* pb = opop + (long long)e * 6;
    float u[6];
    if (gen == 0) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            u[j] = pb[j];
            xv[j] = pb[j];
            xv[6 + j] = 0.0f;
        }
    } else {
        const float* F = ofit + (long long)g * n_out;
        int gb = 0;
        for (int q = 1; q < n_out; ++q)
            if (F[q] < F[gb]) gb = q;
        const float* gbest = opop + ((long long)g * n_out + gb) * 6;
        const Ctr c = make_ctr(key, (uint32_t)g, gen, (uint32_t)i, 0u);
        const uint4 w0 = c.slot(0), w1 = c.slot(1), w2 = c.slot(2);
        const uint32_t r1w[6] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y};
        const uint32_t r2w[6] = {w1.z, w1.w, w2.x, w2.y, w2.z, w2.w};
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const float x = xv[j];
            const float v = 0.729f * xv[6 + j] + 1.49f * uniform24(r1w[j]) * (pb[j] - x) +
                            1.49f * uniform24(r2w[j]) * (gbest[j] - x);
            const float xn = fminf(fmaxf(x + v, c_lb[j]), c_ub[j]);
            xv[6 + j] = v;
            xv[j] = xn;
            u[j] = xn;
        }
    }
    float* th = theta + (long long)e * 6;
    th[0] = u[0];
    th[1] = u[1];
    const float top[4] = {4.f, 4.f, 4.f, 3.f};
#pragma unroll
    for (int j = 2; j < 6; ++j) th[j] = fminf(fmaxf(floorf(u[j]), 1.0f), top[j - 2]);
}

// theta of one evolver vector: F = u1, CR = u2, the categorical genes
// floor(u) clamped to their domains (Alg. 3, decoding).
__device__ __forceinline__ void write_theta(const float (&u)[6], float* th) {
    th[0] = u[0];
    th[1] = u[1];
    const float top[4] = {4.f, 4.f, 4.f, 3.f};
#pragma unroll
    for (int j = 2; j < 6; ++j) th[j] = fminf(fmaxf(floorf(u[j]), 1.0f), top[j - 2]);
}

// CSO evolver (Competitive Swarm Optimizer, Cheng and Jin 2015; the
// supplement's comparison of evolvers).  opop / ofit hold the positions and
// their fitness; trial holds [position to evaluate 6 | velocity 6 | flag] per
// particle.  Generation 0 evaluates the initial swarm (all flagged, v = 0).
// Later generations pair the swarm by a Fisher-Yates permutation (position t
// swaps with int[0, t + 1) from draw slot 3 word 0 of individual t, for
// t = m - 1 down to 1; pairs (pi[2p], pi[2p + 1]), an odd last particle sits
// out).  The fitter particle of a pair (ties to the lower index) is kept; the
// other is flagged and learns from it, with the swarm-mean factor phi = 0:
//   v <- r1 v + r2 (x_w - x_l),  x' = clip(x_l + v),
// r1 / r2 the uniforms of the loser's draw words 0..5 / 6..11 (slot = word / 4).
// One CTA per run; shared memory holds the permutation and the swap targets.
__global__ void k_cso_move(int n_out, Key key, const uint32_t* gen_dev, uint32_t gen_arg,
                           const float* __restrict__ opop, const float* __restrict__ ofit, float* trial,
                           float* theta) {
    extern __shared__ int perm[];
    int* jt = perm + n_out;
    const int g = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const uint32_t gen = gen_dev ? *gen_dev : gen_arg;
    const long long base = (long long)g * n_out;
    auto keep = [&](int i) {  // evaluated as it is; its stored fitness stays
        float* tr = trial + (base + i) * 13;
        float u[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            u[j] = opop[(base + i) * 6 + j];
            tr[j] = u[j];
        }
        tr[12] = 0.f;
        write_theta(u, theta + (base + i) * 6);
    };
    if (gen == 0) {
        for (int i = tid; i < n_out; i += nt) {
            keep(i);
            float* tr = trial + (base + i) * 13;
#pragma unroll
            for (int j = 0; j < 6; ++j) tr[6 + j] = 0.f;
            tr[12] = 1.f;
        }
        return;
    }
    for (int t = tid; t < n_out; t += nt) {
        perm[t] = t;
        jt[t] = t >= 1 ? (int)below(make_ctr(key, (uint32_t)g, gen, (uint32_t)t, 0u).slot(3).x, (uint32_t)(t + 1)) : 0;
    }
    __syncthreads();
    if (tid == 0)
        for (int t = n_out - 1; t >= 1; --t) {
            const int a = perm[t];
            perm[t] = perm[jt[t]];
            perm[jt[t]] = a;
        }
    __syncthreads();
    const int npair = n_out / 2;
    for (int q = tid; q < npair + (n_out & 1); q += nt) {
        if (q == npair) {
            keep(perm[n_out - 1]);
            continue;
        }
        const int a = perm[2 * q], b = perm[2 * q + 1];
        const float fa = ofit[base + a], fb = ofit[base + b];
        const bool a_wins = fa < fb || (fa == fb && a < b);
        const int w = a_wins ? a : b, l = a_wins ? b : a;
        keep(w);
        const Ctr c = make_ctr(key, (uint32_t)g, gen, (uint32_t)l, 0u);
        const uint4 w0 = c.slot(0), w1 = c.slot(1), w2 = c.slot(2);
        const uint32_t r1w[6] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y};
        const uint32_t r2w[6] = {w1.z, w1.w, w2.x, w2.y, w2.z, w2.w};
        float* tr = trial + (base + l) * 13;
        float u[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const float xl = opop[(base + l) * 6 + j], xw = opop[(base + w) * 6 + j];
            const float v = uniform24(r1w[j]) * tr[6 + j] + uniform24(r2w[j]) * (xw - xl);
            const float x = fminf(fmaxf(xl + v, c_lb[j]), c_ub[j]);
            tr[6 + j] = v;
            tr[j] = x;
            u[j] = x;
        }
        tr[12] = 1.f;
        write_theta(u, theta + (base + l) * 6);
    }
}

// CSO selection: a flagged particle takes its evaluated position and
// meta-fitness (NaN as +inf) unconditionally; the others keep theirs.
__global__ void k_cso_select(int n_total, float* opop, float* ofit, const float* __restrict__ trial,
                             const float* __restrict__ meta_fit) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_total) return;
    const float* tr = trial + (long long)e * 13;
    if (tr[12] == 0.f) return;
#pragma unroll
    for (int j = 0; j < 6; ++j) opop[(long long)e * 6 + j] = tr[j];
    const float y = meta_fit[e];
    ofit[e] = isnan(y) ? INFINITY : y;
}

// NES evolver: xNES (Wierstra et al., JMLR 2014) over the 6 genes, search
// distribution N(mu, sigma^2 B B^T), det B = 1.  trial holds per run
// [n_out][z 6 | s 6] (the clipped sample evaluated and its standard-normal
// draw) followed by 96 floats holding the state as doubles: mu[6], sigma,
// B[6][6] row-major.  Generation 0 first sets mu = (lb + ub) / 2 and
// sigma B = diag((ub - lb) / 4) (sigma the geometric mean of the diagonal).
// Sample k: Box-Muller on draw words 2q, 2q + 1 of individual k
// (u1 = ((w >> 8) + 1) 2^-24, u2 = (w >> 8) 2^-24), z = mu + sigma B s,
// evaluated at clip(z).  The update ranks the samples by meta-fitness (NaN
// as +inf, ties to the lower index), weights them by the utilities
// u_r = max(0, ln(lambda/2 + 1) - ln(r + 1)) / sum - 1/lambda and takes the
// natural-gradient step
//   mu += sigma B G_delta,  sigma *= exp(eta G_sigma / 2),  B <- B expm(eta G_B / 2),
// G_delta = sum u s, G_M = sum u (s s^T - I), G_sigma = tr G_M / 6,
// G_B = G_M - G_sigma I, eta = 3 (3 + ln 6) / (5 6 sqrt 6) (the paper's
// defaults, eta_mu = 1).  opop / ofit then hold the samples and their
// meta-fitness.  All of it in FP64, one CTA (a warp) per run.
__host__ __device__ inline long long nes_block(int n_out) { return 12LL * n_out + 96; }

__device__ __forceinline__ double* nes_state(float* trial, int g, int n_out) {
    return reinterpret_cast<double*>(trial + (long long)g * nes_block(n_out) + 12LL * n_out);
}

__global__ void k_nes_sample(int n_out, Key key, const uint32_t* gen_dev, uint32_t gen_arg, float* trial,
                             float* theta) {
    __shared__ double sst[43];
    const int g = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const uint32_t gen = gen_dev ? *gen_dev : gen_arg;
    double* st = nes_state(trial, g, n_out);
    if (gen == 0 && tid == 0) {
        double lg = 0.0;
        for (int j = 0; j < 6; ++j) lg += log((double)(c_ub[j] - c_lb[j]) * 0.25);
        const double sigma = exp(lg / 6.0);
        for (int j = 0; j < 6; ++j) st[j] = 0.5 * ((double)c_lb[j] + (double)c_ub[j]);
        st[6] = sigma;
        for (int r = 0; r < 6; ++r)
            for (int c = 0; c < 6; ++c) st[7 + 6 * r + c] = r == c ? (double)(c_ub[r] - c_lb[r]) * 0.25 / sigma : 0.0;
    }
    __syncthreads();
    for (int q = tid; q < 43; q += nt) sst[q] = st[q];
    __syncthreads();
    for (int k = tid; k < n_out; k += nt) {
        const Ctr c = make_ctr(key, (uint32_t)g, gen, (uint32_t)k, 0u);
        const uint4 w0 = c.slot(0), w1 = c.slot(1);
        const uint32_t w[6] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y};
        double sv[6];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double u1 = (double)((w[2 * q] >> 8) + 1u) * (1.0 / 16777216.0);
            const double u2 = (double)(w[2 * q + 1] >> 8) * (1.0 / 16777216.0);
            const double rad = sqrt(-2.0 * log(u1));
            double sn, cs;
            sincospi(2.0 * u2, &sn, &cs);
            sv[2 * q] = rad * cs;
            sv[2 * q + 1] = rad * sn;
        }
        float* tr = trial + (long long)g * nes_block(n_out) + 12LL * k;
        float u[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            double a = 0.0;
#pragma unroll
            for (int cc = 0; cc < 6; ++cc) a += sst[7 + 6 * r + cc] * sv[cc];
            const double z = fmin(fmax(sst[r] + sst[6] * a, (double)c_lb[r]), (double)c_ub[r]);
            u[r] = (float)z;
            tr[r] = u[r];
            tr[6 + r] = (float)sv[r];
        }
        write_theta(u, theta + ((long long)g * n_out + k) * 6);
    }
}

// exp of a 6 x 6 matrix by scaling and squaring of its Taylor series:
// A / 2^s with infinity norm <= 1/2, 20 terms, then s squarings.
__device__ void expm6(const double* A, double* E) {
    double nrm = 0.0;
    for (int i = 0; i < 6; ++i) {
        double r = 0.0;
        for (int j = 0; j < 6; ++j) r += fabs(A[6 * i + j]);
        nrm = fmax(nrm, r);
    }
    int sq = 0;
    while (nrm > 0.5 && sq < 60) {
        nrm *= 0.5;
        ++sq;
    }
    const double sc = ldexp(1.0, -sq);
    double X[36], T[36], W[36];
    for (int i = 0; i < 36; ++i) {
        X[i] = A[i] * sc;
        T[i] = (i % 7 == 0) ? 1.0 : 0.0;
        E[i] = T[i];
    }
    for (int k = 1; k <= 20; ++k) {
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double a = 0.0;
                for (int q = 0; q < 6; ++q) a += T[6 * i + q] * X[6 * q + j];
                W[6 * i + j] = a / k;
            }
        for (int i = 0; i < 36; ++i) {
            T[i] = W[i];
            E[i] += W[i];
        }
    }
    for (int r = 0; r < sq; ++r) {
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double a = 0.0;
                for (int q = 0; q < 6; ++q) a += E[6 * i + q] * E[6 * q + j];
                W[6 * i + j] = a;
            }
        for (int i = 0; i < 36; ++i) E[i] = W[i];
    }
}

__global__ void __launch_bounds__(32) k_nes_update(int n_out, float* opop, float* ofit, float* trial,
                                                   const float* __restrict__ meta_fit) {
    const int g = blockIdx.x, lane = threadIdx.x;
    const long long base = (long long)g * n_out;
    const float* tg = trial + (long long)g * nes_block(n_out);
    double* st = nes_state(trial, g, n_out);
    const double lam = (double)n_out, top = log(lam * 0.5 + 1.0);
    double den = 0.0;
    for (int r = lane; r < n_out; r += 32) den += fmax(0.0, top - log(r + 1.0));
    den = warp_sum(den);
    double gd[6] = {0, 0, 0, 0, 0, 0}, gm[21] = {0};  // G_delta, upper triangle of G_M
    for (int k = lane; k < n_out; k += 32) {
        float yk = meta_fit[base + k];
        if (isnan(yk)) yk = INFINITY;
        int rank = 0;
        for (int j = 0; j < n_out; ++j) {
            float yj = meta_fit[base + j];
            if (isnan(yj)) yj = INFINITY;
            rank += (yj < yk || (yj == yk && j < k)) ? 1 : 0;
        }
        const double uk = fmax(0.0, top - log(rank + 1.0)) / den - 1.0 / lam;
        double sv[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            sv[i] = (double)tg[12LL * k + 6 + i];
            gd[i] += uk * sv[i];
        }
        int t = 0;
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = i; j < 6; ++j, ++t) gm[t] += uk * (sv[i] * sv[j] - (i == j ? 1.0 : 0.0));
#pragma unroll
        for (int i = 0; i < 6; ++i) opop[(base + k) * 6 + i] = tg[12LL * k + i];
        ofit[base + k] = yk;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) gd[i] = warp_sum(gd[i]);
#pragma unroll
    for (int t = 0; t < 21; ++t) gm[t] = warp_sum(gm[t]);
    if (lane != 0) return;
    const double eta = 3.0 * (3.0 + log(6.0)) / (5.0 * 6.0 * sqrt(6.0));
    double GM[36];
    int t = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j, ++t) GM[6 * i + j] = GM[6 * j + i] = gm[t];
    const double gs = (GM[0] + GM[7] + GM[14] + GM[21] + GM[28] + GM[35]) / 6.0;
    double H[36], Ex[36], Bn[36];
    for (int i = 0; i < 36; ++i) H[i] = 0.5 * eta * (GM[i] - ((i % 7 == 0) ? gs : 0.0));
    expm6(H, Ex);
    const double sigma = st[6];
    for (int i = 0; i < 6; ++i) {
        double a = 0.0;
        for (int j = 0; j < 6; ++j) a += st[7 + 6 * i + j] * gd[j];
        st[i] += sigma * a;
    }
    st[6] = sigma * exp(0.5 * eta * gs);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double a = 0.0;
            for (int q = 0; q < 6; ++q) a += st[7 + 6 * i + q] * Ex[6 * q + j];
            Bn[6 * i + j] = a;
        }
    for (int i = 0; i < 36; ++i) st[7 + i] = Bn[i];
}

// Alg. 3 selection; tstride is the trial's floats per vector (6 for DE, 12
// for PSO, whose first 6 are the position).
__global__ void k_outer_select(int n_total, float* opop, float* ofit, const float* __restrict__ trial,
                               const float* __restrict__ meta_fit, int tstride) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_total) return;
    float y = meta_fit[e];
    if (isnan(y)) y = INFINITY;
    if (y <= ofit[e]) {
#pragma unroll
        for (int j = 0; j < 6; ++j) opop[(long long)e * 6 + j] = trial[(long long)e * tstride + j];
        ofit[e] = y;
    }
}

cudaError_t launch_outer_init(int n_groups, int n_out, Key key, float* opop, float* ofit, cudaStream_t st) {
    const int n = n_groups * n_out;
    k_outer_init<<<(n + 127) / 128, 128, 0, st>>>(n, n_out, key, opop, ofit);
    return cudaGetLastError();
}

cudaError_t launch_outer_trial(int n_groups, int n_out, Key key, const uint32_t* gen_dev, uint32_t gen,
                               const float* opop, float* trial, float* theta, cudaStream_t st) {
    const int n = n_groups * n_out;
    k_outer_trial<<<(n + 127) / 128, 128, 0, st>>>(n, n_out, key, gen_dev, gen, opop, trial, theta);
    return cudaGetLastError();
}

cudaError_t launch_outer_select(int n_groups, int n_out, float* opop, float* ofit, const float* trial,
                                const float* meta_fit, int tstride, cudaStream_t st) {
    const int n = n_groups * n_out;
    k_outer_select<<<(n + 127) / 128, 128, 0, st>>>(n, opop, ofit, trial, meta_fit, tstride);
    return cudaGetLastError();
}

cudaError_t launch_cso_move(int n_groups, int n_out, Key key, const uint32_t* gen_dev, uint32_t gen,
                            const float* opop, const float* ofit, float* trial, float* theta, cudaStream_t st) {
    if (n_groups <= 0) return cudaSuccess;
    k_cso_move<<<n_groups, 128, 2 * sizeof(int) * (size_t)n_out, st>>>(n_out, key, gen_dev, gen, opop, ofit, trial,
                                                                      theta);
    return cudaGetLastError();
}

cudaError_t launch_cso_select(int n_groups, int n_out, float* opop, float* ofit, const float* trial,
                              const float* meta_fit, cudaStream_t st) {
    const int n = n_groups * n_out;
    if (n <= 0) return cudaSuccess;
    k_cso_select<<<(n + 127) / 128, 128, 0, st>>>(n, opop, ofit, trial, meta_fit);
    return cudaGetLastError();
}

cudaError_t launch_nes_sample(int n_groups, int n_out, Key key, const uint32_t* gen_dev, uint32_t gen, float* trial,
                              float* theta, cudaStream_t st) {
    if (n_groups <= 0) return cudaSuccess;
    k_nes_sample<<<n_groups, 128, 0, st>>>(n_out, key, gen_dev, gen, trial, theta);
    return cudaGetLastError();
}

cudaError_t launch_nes_update(int n_groups, int n_out, float* opop, float* ofit, float* trial, const float* meta_fit,
                              cudaStream_t st) {
    if (n_groups <= 0) return cudaSuccess;
    k_nes_update<<<n_groups, 32, 0, st>>>(n_out, opop, ofit, trial, meta_fit);
    return cudaGetLastError();
}

cudaError_t launch_pso_move(int n_groups, int n_out, Key key, const uint32_t* gen_dev, uint32_t gen,
                            const float* opop, const float* ofit, float* trial, float* theta, cudaStream_t st) {
    const int n = n_groups * n_out;
    k_pso_move<<<(n + 127) / 128, 128, 0, st>>>(n, n_out, key, gen_dev, gen, opop, ofit, trial, theta);
    return cudaGetLastError();
}

}  // namespace metade
