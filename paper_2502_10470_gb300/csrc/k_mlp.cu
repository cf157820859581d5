// k_mlp.cu -- the MLP regression objective (6), a neuroevolution-like
// large-D problem: its fixed inputs and teacher targets, and the batched path
// for its executors.
//
// k_mlp_inputs    the 256 x 16 inputs, uniform in [-1, 1] (counter-based draws)
// k_mlp_targets   teacher outputs of one problem, by the same FP32 forward pass
//                 the evaluation uses (so f(teacher) = 0 exactly)
// k_fused_mlp     one CTA (256 threads) per executor runs all fused
//                 generations: trials by warps (the PDE step of every other
//                 kernel), then each individual's f with thread n evaluating
//                 input n (the parameters in shared memory, read as
//                 broadcasts; the thread's input row in registers), a block
//                 sum, then greedy selection on the FP32 values
#include "block.cuh"
#include "internal.h"

namespace metade {

__global__ void k_mlp_inputs(float* X) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kMlpN * kMlpIn) return;
    const int n = e / kMlpIn, k = e - n * kMlpIn;
    const uint4 w = philox(0u, 0u, (uint32_t)n, (uint32_t)(k / 4), make_key(0, kTagData));
    X[e] = 2.0f * uniform24(word_of(w, k & 3)) - 1.0f;
}

__global__ void k_mlp_targets(const float* __restrict__ X, const float* __restrict__ teacher, int h, float* Y) {
    const int n = threadIdx.x;  // one block of kMlpN threads
    float x[kMlpIn], y[kMlpOut];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) x[k] = X[n * kMlpIn + k];
    mlp_forward<float>(h, teacher, x, y);
    Y[2 * n] = y[0];
    Y[2 * n + 1] = y[1];
}

__global__ void __launch_bounds__(256) k_fused_mlp(StepArgs a, const int* __restrict__ work, int n_work,
                                                   float* uscr, const float* __restrict__ mlp_x,
                                                   const float* __restrict__ mlp_y, int max_np, int max_dpad) {
    extern __shared__ __align__(16) float sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;  // thread tid evaluates input tid
    float* f = sm;
    float* fu = f + max_np;
    int* topk = reinterpret_cast<int*>(fu + max_np);  // pbest ranks; selection: accept flags
    int* red = topk + max_np;                         // 64 words
    float* th = sm + ((3 * max_np + 64 + 3) & ~3);    // parameters of the individual being evaluated
    float* db = th + max_dpad;                        // per warp: u - o of the trial kernel
    float x[kMlpIn];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) x[k] = mlp_x[tid * kMlpIn + k];
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const int k = work[w];
        const InstDesc d = a.desc[k];
        const Strat st = load_strat(a.theta + 6 * k, d.np);
        if (!st.ok) {
            if (tid == 0) set_status(a.status, 1);
            continue;
        }
        const int np = d.np, dim = d.dim, dp = d.dpad, nbr = dp >> 2, h = mlp_hidden(dim);
        const float y0 = mlp_y[d.aux + 2 * tid], y1 = mlp_y[d.aux + 2 * tid + 1];
        const uint32_t epoch = a.epoch_dev ? *a.epoch_dev : a.epoch;
        float* X = a.pop + d.pop_off;
        float* Ug = uscr + d.pop_off;
        const float* o = a.shift + d.shift_off;
        for (int i = tid; i < np; i += blockDim.x) f[i] = a.fit[d.fit_off + i];
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
            // trials, warp per individual, into the scratch population
            for (int i = warp; i < np; i += blockDim.x >> 5) {
                const Ctr c = make_ctr(a.key, (uint32_t)d.stream, gen, (uint32_t)i, epoch);
                Indiv v;
                indiv_setup(st, c, i, np, dim, d.kp, pb ? topk : nullptr, best, v);
                const int L = st.cs == 2 ? exp_length(c, dim, st.cri) : 0;
                warp_trial(st, c, v, i, dim, L, X, dp, o, a.lo, a.hi, Ug + (long long)i * dp,
                           db + (size_t)warp * max_dpad);
                __syncwarp();
            }
            __syncthreads();
            // f of every trial: thread n runs input n, then a block sum
            for (int i = 0; i < np; ++i) {
                for (int e = tid; e < dim; e += blockDim.x) th[e] = Ug[(long long)i * dp + e];
                __syncthreads();
                float y[kMlpOut];
                mlp_forward<float>(h, th, x, y);
                const float e0 = y[0] - y0, e1 = y[1] - y1;
                float s = warp_sum(fmaf(e0, e0, e1 * e1));
                if (lane == 0) reinterpret_cast<float*>(red)[warp] = s;
                __syncthreads();
                if (tid == 0) {
                    float t = 0.0f;
                    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += reinterpret_cast<float*>(red)[q];
                    fu[i] = nan_to_inf(t * (1.0f / (kMlpN * kMlpOut)));
                }
                __syncthreads();
            }
            // greedy selection on the FP32 values (no difference form exists for this objective)
            int* acc = topk;
            for (int i = tid; i < np; i += blockDim.x) {
                const float fn = fu[i];
                const int take = fn <= f[i] ? 1 : 0;
                if (take) f[i] = fn;
                acc[i] = take;
            }
            __syncthreads();
            for (int e = tid; e < np * nbr; e += blockDim.x) {
                const int i = e / nbr, q = e - i * nbr;
                if (acc[i])
                    *reinterpret_cast<float4*>(X + (long long)i * dp + 4 * q) =
                        *reinterpret_cast<const float4*>(Ug + (long long)i * dp + 4 * q);
            }
            __syncthreads();
        }
        for (int i = tid; i < np; i += blockDim.x) a.fit[d.fit_off + i] = f[i];
        const int b = block_argmin(f, np, red);
        if (tid == 0 && a.best_f) a.best_f[k] = f[b];
        if (tid == 0 && a.best_i) a.best_i[k] = b;
        __syncthreads();
    }
}

size_t fused_smem_mlp(int max_np, int max_dpad) {
    size_t words = (3 * (size_t)max_np + 64 + 3) & ~(size_t)3;
    words += (size_t)max_dpad;      // parameters being evaluated
    words += (size_t)8 * max_dpad;  // per-warp trial scratch (8 warps)
    return words * sizeof(float);
}

cudaError_t launch_fused_mlp(const StepArgs& a, const int* work, int n_work, const FusedPlan& p, float* uscr,
                             const float* mlp_x, const float* mlp_y, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    if (p.threads != kMlpN) return cudaErrorInvalidValue;  // thread n evaluates input n
    cudaError_t e = cudaFuncSetAttribute(k_fused_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    k_fused_mlp<<<p.grid, p.threads, p.smem, st>>>(a, work, n_work, uscr, mlp_x, mlp_y, p.max_np, p.max_dpad);
    return cudaGetLastError();
}

cudaError_t launch_mlp_inputs(float* X, cudaStream_t st) {
    k_mlp_inputs<<<(kMlpN * kMlpIn + 255) / 256, 256, 0, st>>>(X);
    return cudaGetLastError();
}

cudaError_t launch_mlp_targets(const float* X, const float* teacher, int h, float* Y, cudaStream_t st) {
    k_mlp_targets<<<1, kMlpN, 0, st>>>(X, teacher, h, Y);
    return cudaGetLastError();
}

}  // namespace metade
