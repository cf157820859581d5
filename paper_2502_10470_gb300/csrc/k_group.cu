// k_group.cu -- batched path for 32 < D <= 256: k_fused_group<S>.
//
// One CTA per executor runs all fused generations (like k_fused_small), but
// an individual is handled by a group of S adjacent lanes (S = 2, 4, 8) that
// split the coordinates: lane s owns the 4-coordinate chunks
// [s*CH, (s+1)*CH) of its individual.  Each lane builds its chunks of the
// trial (draws are recomputed by every lane of the group, crossover uniforms
// only for its own chunks), keeps its part of d = u - o in registers, and
// computes partial dot products z_r = sum_{c in its chunks} R[r][c] d_c for
// a block of S rows at a time; a butterfly reduce-scatter over the group
// leaves lane s with the complete z of row r0 + s.  Objective terms are
// accumulated per lane and combined across the group at the end (group sums,
// a group scan for the Schwefel prefix sums, neighbour shuffles for
// Rosenbrock, (P, Q) product pairs for Griewank).  The exponential
// crossover length is the first failing uniform over all lanes' chunks (a
// group min) instead of a sequential scan.  Near ties are decided in
// selection by the group itself with the FP32 difference form.
#include "block.cuh"
#include "group_obj.cuh"
#include "internal.h"

namespace metade {

namespace {

constexpr int kCMAX = 32;  // coordinates per lane (8 chunks)

// Butterfly reduce-scatter over a group of S lanes: on entry lane s holds
// partial sums p[0..S) of S rows; on exit lane s returns the full sum of row
// s.  At each level the lane keeps the half of its values whose row index
// has the lane's bit, and adds the partner's copy of that half.
template <int S>
__device__ __forceinline__ float reduce_scatter(float (&p)[S], int s) {
#pragma unroll
    for (int half = S / 2; half >= 1; half >>= 1) {
        const bool upper = (s & half) != 0;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const float send = upper ? p[j] : p[j + half];
            const float keep = upper ? p[j + half] : p[j];
            p[j] = keep + __shfl_xor_sync(kFull, send, half);
        }
    }
    return p[0];
}


// f(u) - f(x) of one individual by its group of S lanes (selection ties):
// x - o and u - x for the lane's chunks in registers, both rotations by the
// same column-split partial sums and reduce-scatter as the trial evaluation,
// then the difference forms (see device.cuh) per row and a group combine.
// Every lane returns the value.
template <int S, bool RS>
__device__ __forceinline__ float group_diff(int obj, int dim, int dp, int CH, int c0, int s, const float* R,
                                            const float* xi, const float* ui, const float* o) {
    float dx[kCMAX], dl[kCMAX];
#pragma unroll
    for (int q = 0; q < kCMAX / 4; ++q) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = c0 + 4 * q + t;
            const bool in = q < CH && j < dim;
            const float xv = in ? xi[j] : 0.f;
            dx[4 * q + t] = in ? xv - o[j] : 0.f;
            dl[4 * q + t] = in ? ui[j] - xv : 0.f;
        }
    }
    GroupDiff g;
    for (int r0 = 0; r0 < dim; r0 += S) {
        float pa[S], pb[S];
#pragma unroll
        for (int b = 0; b < S; ++b) {
            const int r = r0 + b;
            float za = 0.f, zb = 0.f;
            if (r < dim) {
                const float* row = R + (long long)r * dp + c0;
#pragma unroll
                for (int q = 0; q < kCMAX / 4; ++q) {
                    if (q < CH && c0 + 4 * q < dp) {
                        const float4* src = reinterpret_cast<const float4*>(row + 4 * q);
                        const float4 rr = RS ? *src : __ldg(src);
                        za = fmaf(rr.x, dx[4 * q + 0], za);
                        za = fmaf(rr.y, dx[4 * q + 1], za);
                        za = fmaf(rr.z, dx[4 * q + 2], za);
                        za = fmaf(rr.w, dx[4 * q + 3], za);
                        zb = fmaf(rr.x, dl[4 * q + 0], zb);
                        zb = fmaf(rr.y, dl[4 * q + 1], zb);
                        zb = fmaf(rr.z, dl[4 * q + 2], zb);
                        zb = fmaf(rr.w, dl[4 * q + 3], zb);
                    }
                }
            }
            pa[b] = za;
            pb[b] = zb;
        }
        const float z = reduce_scatter<S>(pa, s), dz = reduce_scatter<S>(pb, s);
        group_diff_push<S>(obj, g, z, dz, r0, s, dim);
    }
    return group_diff_finish<S>(obj, g, dim);
}

}  // namespace

template <int S, bool RS>
__global__ void __launch_bounds__(512) k_fused_group(StepArgs a, const int* __restrict__ work, int n_work,
                                                     float* uscr, int pop_smem, int max_np, int max_dpad) {
    constexpr int rot_smem = RS ? 1 : 0;
    extern __shared__ __align__(16) float sm[];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    const int s = lane & (S - 1);           // lane within the group
    const int gi = tid / S, ng = nt / S;    // group index, groups per CTA
    float* f = sm;
    float* fu = f + max_np;
    int* topk = reinterpret_cast<int*>(fu + max_np);
    int* ties = topk + max_np;              // reserved
    int* red = ties + max_np;               // 64 words (block reductions)
    float* Rs = sm + ((4 * max_np + 64 + 3) & ~3);
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const int k = work[w];
        const InstDesc d = a.desc[k];
        const Strat st = load_strat(a.theta + 6 * k, d.np);
        if (!st.ok) {
            if (tid == 0) set_status(a.status, 1);
            continue;
        }
        const int np = d.np, dim = d.dim, dp = d.dpad, nch = dp >> 2;
        const float band = tie_band(dim);
        const int CH = (nch + S - 1) / S;   // chunks per lane (<= kCMAX / 4 by the planner)
        const int c0 = s * CH * 4;          // first coordinate of this lane
        const uint32_t epoch = a.epoch_dev ? *a.epoch_dev : a.epoch;
        float* const Xg = a.pop + d.pop_off;
        float* X = Xg;
        float* Ug = uscr + d.pop_off;
        const float* o = a.shift + d.shift_off;
        const float* R = a.rot + d.rot_off;  // row-major [dim][dp]
        if (rot_smem) {
            for (int e = tid; e < dim * (dp >> 2); e += nt)
                reinterpret_cast<float4*>(Rs)[e] = reinterpret_cast<const float4*>(R)[e];
            R = Rs;
        }
        if (pop_smem) {  // after the R region (sized for the bucket's widest executor)
            X = Rs + (rot_smem ? (size_t)max_dpad * max_dpad : 0);
            for (int e = tid; e < np * (dp >> 2); e += nt)
                reinterpret_cast<float4*>(X)[e] = reinterpret_cast<const float4*>(Xg)[e];
        }
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
            for (int base = 0; base < np; base += ng) {
                const int i0 = base + gi;
                const bool act = i0 < np;
                const int i = act ? i0 : np - 1;  // inactive groups shadow a valid individual, writes skipped
                const Ctr c = make_ctr(a.key, (uint32_t)d.stream, gen, (uint32_t)i, epoch);
                Indiv v;
                indiv_setup(st, c, i, np, dim, d.kp, pb ? topk : nullptr, best, v);
                // exponential length: first failing uniform among all lanes' chunks
                int L = 0;
                if (st.cs == 2) {
                    int first = dim;  // index of the first uniform >= CR (words 0..dim-2)
                    for (int q = 0; q < CH; ++q) {
                        const int ch = s * CH + q;
                        if (4 * ch >= dim - 1) break;
                        const uint4 wv = c.slot(4 + (uint32_t)ch);
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int l = 4 * ch + t;
                            if (l < dim - 1 && l < first && (word_of(wv, t) >> 8) >= st.cri) first = l;
                        }
                        if (first < dim) break;
                    }
                    first = gmin<S>(first);
                    L = first < dim - 1 ? first + 1 : dim;
                }
                // trial chunks of this lane; d = u - o kept in registers
                float dreg[kCMAX];
                const float F = st.F, K = (float)v.kraw * (1.0f / 16777216.0f);
                const float* xl = X + (long long)v.ibl * dp;
                const float* xr = X + (long long)v.ibr * dp;
                const float* xi = X + (long long)i * dp;
                const bool dir = st.bl != st.br;
#pragma unroll
                for (int q = 0; q < kCMAX / 4; ++q) {
                    const int j4 = c0 + 4 * q;
                    if (q < CH && j4 < dp) {
                        const float4 av = *reinterpret_cast<const float4*>(xl + j4);
                        const float4 bv = *reinterpret_cast<const float4*>(xr + j4);
                        const float4 xv = *reinterpret_cast<const float4*>(xi + j4);
                        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
                        for (int t = 0; t < st.dn; ++t) {
                            const float4 pp =
                                *reinterpret_cast<const float4*>(X + (long long)diff_plus(v, st.a, t) * dp + j4);
                            const float4 mm =
                                *reinterpret_cast<const float4*>(X + (long long)diff_minus(v, st.a, t) * dp + j4);
                            sum.x += pp.x - mm.x; sum.y += pp.y - mm.y; sum.z += pp.z - mm.z; sum.w += pp.w - mm.w;
                        }
                        const uint4 wv = (st.cs == 1) ? c.slot(4 + (uint32_t)(j4 >> 2)) : make_uint4(0, 0, 0, 0);
                        const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
                        const float x4[4] = {xv.x, xv.y, xv.z, xv.w}, s4[4] = {sum.x, sum.y, sum.z, sum.w};
                        float u4[4];
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int j = j4 + t;
                            float vj = a4[t];
                            if (dir) vj += F * (b4[t] - a4[t]);
                            vj += F * s4[t];
                            float u;
                            if (st.cs == 3) {
                                u = x4[t] + K * (vj - x4[t]);
                            } else {
                                bool take;
                                if (st.cs == 1) {
                                    take = ((word_of(wv, t) >> 8) < st.cri) || (j == v.jrand);
                                } else {
                                    int off = j - v.nstart;
                                    if (off < 0) off += dim;
                                    take = off < L;
                                }
                                u = take ? vj : x4[t];
                            }
                            u = fminf(fmaxf(u, a.lo), a.hi);
                            if (j >= dim) u = 0.0f;
                            u4[t] = u;
                            dreg[4 * q + t] = (j < dim) ? (u - o[j]) : 0.0f;
                        }
                        if (act)
                            *reinterpret_cast<float4*>(Ug + (long long)i * dp + j4) =
                                make_float4(u4[0], u4[1], u4[2], u4[3]);
                    } else {
#pragma unroll
                        for (int t = 0; t < 4; ++t) dreg[4 * q + t] = 0.0f;
                    }
                }
                // rotation by row blocks of S, objective per lane
                GroupObj acc;
                const int obj = d.obj;
                unsigned okm = 0;  // chunks this lane owns inside the row
#pragma unroll
                for (int q = 0; q < kCMAX / 4; ++q)
                    if (q < CH && c0 + 4 * q < dp) okm |= 1u << q;
                const float* Rl = R + c0;
                for (int r0 = 0; r0 < dim; r0 += S) {
                    float p[S];
                    const int nb = min(S, dim - r0);
                    const float* rb = Rl + (size_t)r0 * dp;
#pragma unroll
                    for (int b = 0; b < S; ++b) p[b] = 0.f;
#pragma unroll
                    for (int q = 0; q < kCMAX / 4; ++q) {
                        if (okm & (1u << q)) {
                            const float d0 = dreg[4 * q], d1 = dreg[4 * q + 1], d2 = dreg[4 * q + 2],
                                        d3 = dreg[4 * q + 3];
#pragma unroll
                            for (int b = 0; b < S; ++b) {
                                if (b < nb) {
                                    const float4* src = reinterpret_cast<const float4*>(rb + (size_t)b * dp + 4 * q);
                                    const float4 rr = RS ? *src : __ldg(src);
                                    p[b] = fmaf(rr.x, d0, p[b]);
                                    p[b] = fmaf(rr.y, d1, p[b]);
                                    p[b] = fmaf(rr.z, d2, p[b]);
                                    p[b] = fmaf(rr.w, d3, p[b]);
                                }
                            }
                        }
                    }
                    const float z = reduce_scatter<S>(p, s);  // full z of row r0 + s
                    group_obj_push<S>(obj, acc, z, r0, s, dim);
                }
                const float fval = group_obj_finish<S>(obj, acc, dim);
                if (act && s == 0) fu[i] = nan_to_inf(fval);
            }
            __syncthreads();
            // selection by groups; near ties decided by the group on the difference form
            for (int base = 0; base < np; base += ng) {
                const int i0 = base + gi;
                const bool act = i0 < np;
                const int i = act ? i0 : np - 1;
                float* Xi = X + (long long)i * dp;
                const float* Ui = Ug + (long long)i * dp;
                const float fx = f[i];
                float fn = fu[i];
                bool tie = near_tie(fn, fx, band);
                bool diff = false;
                for (int q = 0; q < CH; ++q) {
                    const int j4 = c0 + 4 * q;
                    if (j4 >= dp) break;
                    const float4 uu = *reinterpret_cast<const float4*>(Ui + j4);
                    const float4 xx = *reinterpret_cast<const float4*>(Xi + j4);
                    diff = diff || uu.x != xx.x || uu.y != xx.y || uu.z != xx.z || uu.w != xx.w;
                }
                diff = gany<S>(diff);
                if (tie && !diff) {
                    tie = false;
                    fn = fx;  // the trial is the target
                }
                tie = tie && act;
                bool take = act && fn <= fx;
                if (__any_sync(kFull, tie)) {  // whole warp runs it; only tie groups use the result
                    const float df = group_diff<S, RS>(d.obj, dim, dp, CH, c0, s, R, Xi, Ui, o);
                    if (tie) {
                        take = df <= 0.0f;
                        fn = fx + df;
                    }
                }
                if (take) {
                    for (int q = 0; q < CH; ++q) {
                        const int j4 = c0 + 4 * q;
                        if (j4 >= dp) break;
                        *reinterpret_cast<float4*>(Xi + j4) = *reinterpret_cast<const float4*>(Ui + j4);
                    }
                    if (s == 0) f[i] = fn;
                }
            }
            __syncthreads();
        }
        if (pop_smem)
            for (int e = tid; e < np * (dp >> 2); e += nt)
                reinterpret_cast<float4*>(Xg)[e] = reinterpret_cast<const float4*>(X)[e];
        for (int i = tid; i < np; i += nt) a.fit[d.fit_off + i] = f[i];
        const int b = block_argmin(f, np, red);
        if (tid == 0 && a.best_f) a.best_f[k] = f[b];
        if (tid == 0 && a.best_i) a.best_i[k] = b;
        __syncthreads();
    }
}

// Lanes per individual for a row length: each lane holds at most kCMAX coordinates.
int group_lanes_for(int dpad) {
    const int nch = dpad >> 2;
    for (int S = 2; S <= 8; S <<= 1)
        if ((nch + S - 1) / S <= kCMAX / 4) return S;
    return 0;
}

size_t fused_smem_group(int max_np, int max_dpad, int threads, bool rot_in_smem, bool pop_in_smem) {
    (void)threads;
    size_t words = (4 * (size_t)max_np + 64 + 3) & ~(size_t)3;
    if (rot_in_smem) words += (size_t)max_dpad * max_dpad;
    if (pop_in_smem) words += (size_t)max_np * max_dpad;
    return words * sizeof(float);
}

template <int S, bool RS>
static cudaError_t launch_group_t(const StepArgs& a, const int* work, int n_work, const FusedPlan& p, float* uscr,
                                  cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_fused_group<S, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    k_fused_group<S, RS><<<p.grid, p.threads, p.smem, st>>>(a, work, n_work, uscr, p.pop_smem, p.max_np, p.max_dpad);
    return cudaGetLastError();
}

cudaError_t launch_fused_group(const StepArgs& a, const int* work, int n_work, const FusedPlan& p, float* uscr,
                               cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    const bool rs = p.rot_smem != 0;
    switch (p.dmax) {  // dmax holds S for this kernel kind
    case 2: return rs ? launch_group_t<2, true>(a, work, n_work, p, uscr, st) : launch_group_t<2, false>(a, work, n_work, p, uscr, st);
    case 4: return rs ? launch_group_t<4, true>(a, work, n_work, p, uscr, st) : launch_group_t<4, false>(a, work, n_work, p, uscr, st);
    case 8: return rs ? launch_group_t<8, true>(a, work, n_work, p, uscr, st) : launch_group_t<8, false>(a, work, n_work, p, uscr, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace metade
