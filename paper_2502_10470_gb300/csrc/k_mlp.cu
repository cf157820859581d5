// k_mlp.cu -- the MLP regression objective (6), a neuroevolution-like
// large-D problem: its fixed inputs and teacher targets, and the batched path
// for its executors, one generation of all of them per four launches:
//
// k_mlp_inputs    the 256 x 16 inputs, uniform in [-1, 1] (counter-based draws)
// k_mlp_targets   teacher outputs of one problem, by the same FP32 forward pass
//                 the evaluation uses (so f(teacher) = 0 exactly)
// k_mlp_prologue  best and pbest pool per executor (block per executor)
// k_mlp_trial     trial rows, warp per individual (the PDE step of every
//                 other kernel), into the scratch population
// k_mlp_eval      f of every trial (and of the initial population), CTA of
//                 128 threads per individual: thread n runs inputs n and
//                 n + 128 together, so every weight load (a shared-memory
//                 broadcast) feeds both; the input rows are in registers;
//                 then a block sum
// k_mlp_select    greedy selection on the FP32 values, warp per individual
//
// Executor k's individuals are rows InstDesc.tc_row .. tc_row + NP - 1 of the
// MLP row list.
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

__global__ void k_mlp_prologue(StepArgs a, const int* __restrict__ execs, int* topk_all) {
    const int k = execs[blockIdx.x];
    const InstDesc d = a.desc[k];
    const Strat s = load_strat(a.theta + 6 * k, d.np);
    if (!s.ok) {
        if (threadIdx.x == 0) set_status(a.status, 1);
        return;
    }
    block_topk_staged(a.fit + d.fit_off, d.np, d.kp, topk_all + d.fit_off);  // topk[0] is the best
}

__global__ void __launch_bounds__(256) k_mlp_trial(StepArgs a, const int* __restrict__ row_exec, int n_rows,
                                                   const int* __restrict__ topk_all, float* uscr, int ws) {
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
    warp_trial(s, c, v, i, d.dim, L, a.pop + d.pop_off, d.dpad, a.shift + d.shift_off, a.lo, a.hi,
               uscr + d.pop_off + (long long)i * d.dpad, smt + (size_t)warp * ws);
}

__global__ void __launch_bounds__(kMlpN / 2) k_mlp_eval(const InstDesc* __restrict__ desc,
                                                       const int* __restrict__ row_exec,
                                                       const float* __restrict__ uscr, const float* __restrict__ mlp_x,
                                                       const float* __restrict__ mlp_y, float* fu) {
    extern __shared__ __align__(16) float th[];  // parameters of this row's trial
    __shared__ float part[kMlpN / 64];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;  // thread tid runs inputs tid, tid + 128
    const int nb = tid + kMlpN / 2;
    const int r = blockIdx.x;
    const InstDesc d = desc[row_exec[r]];
    const int i = r - d.tc_row, h = mlp_hidden(d.dim);
    const float* u = uscr + d.pop_off + (long long)i * d.dpad;
    for (int e = tid; e < d.dim; e += blockDim.x) th[e] = u[e];
    float xa[kMlpIn], xb[kMlpIn];
#pragma unroll
    for (int q = 0; q < kMlpIn; ++q) {
        xa[q] = mlp_x[tid * kMlpIn + q];
        xb[q] = mlp_x[nb * kMlpIn + q];
    }
    __syncthreads();
    float ya[kMlpOut], yb[kMlpOut];
    mlp_forward2(h, th, xa, xb, ya, yb);
    const float ea0 = ya[0] - mlp_y[d.aux + 2 * tid], ea1 = ya[1] - mlp_y[d.aux + 2 * tid + 1];
    const float eb0 = yb[0] - mlp_y[d.aux + 2 * nb], eb1 = yb[1] - mlp_y[d.aux + 2 * nb + 1];
    const float s = warp_sum(fmaf(ea0, ea0, ea1 * ea1) + fmaf(eb0, eb0, eb1 * eb1));
    if (lane == 0) part[warp] = s;
    __syncthreads();
    if (tid == 0) {
        float t = 0.0f;
        for (int q = 0; q < kMlpN / 64; ++q) t += part[q];
        fu[d.fit_off + i] = nan_to_inf(t * (1.0f / (kMlpN * kMlpOut)));
    }
}

__global__ void __launch_bounds__(256) k_mlp_select(StepArgs a, const int* __restrict__ row_exec, int n_rows,
                                                    const float* __restrict__ uscr, const float* __restrict__ fu) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + warp;
    if (r >= n_rows) return;
    const int k = row_exec[r];
    const InstDesc d = a.desc[k];
    if (!load_strat(a.theta + 6 * k, d.np).ok) return;
    const int i = r - d.tc_row;
    const float fn = fu[d.fit_off + i];
    if (fn <= a.fit[d.fit_off + i]) {  // FP32 values decide: the objective has no difference form
        float* X = a.pop + d.pop_off + (long long)i * d.dpad;
        const float* U = uscr + d.pop_off + (long long)i * d.dpad;
        for (int j = lane * 4; j < d.dpad; j += 128)
            *reinterpret_cast<float4*>(X + j) = *reinterpret_cast<const float4*>(U + j);
        if (lane == 0) a.fit[d.fit_off + i] = fn;
    }
}

cudaError_t launch_mlp_generation(const StepArgs& a, const MlpPlan& p, cudaStream_t st) {
    if (p.n_rows <= 0) return cudaSuccess;
    k_mlp_prologue<<<p.n_exec, 256, 0, st>>>(a, p.execs, p.topk_all);
    const int blocks = (p.n_rows + 7) / 8;
    const size_t smem_t = (size_t)8 * p.max_dpad * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_trial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t);
    if (e != cudaSuccess) return e;
    k_mlp_trial<<<blocks, 256, smem_t, st>>>(a, p.row_exec, p.n_rows, p.topk_all, p.uscr, p.max_dpad);
    const size_t smem_e = (size_t)p.max_dpad * sizeof(float);
    if (p.tc) {
        e = launch_mlp_eval_tc(a.desc, p, p.uscr, p.fu, a.status, st);
        if (e != cudaSuccess) return e;
    } else {
        e = cudaFuncSetAttribute(k_mlp_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_e);
        if (e != cudaSuccess) return e;
        k_mlp_eval<<<p.n_rows, kMlpN / 2, smem_e, st>>>(a.desc, p.row_exec, p.uscr, p.x, p.y, p.fu);
    }
    k_mlp_select<<<blocks, 256, 0, st>>>(a, p.row_exec, p.n_rows, p.uscr, p.fu);
    return cudaGetLastError();
}

cudaError_t launch_mlp_eval(const InstDesc* desc, const MlpPlan& p, const float* rows, float* f_out, int* status,
                            cudaStream_t st) {
    if (p.n_rows <= 0) return cudaSuccess;
    if (p.tc) return launch_mlp_eval_tc(desc, p, rows, f_out, status, st);
    const size_t smem_e = (size_t)p.max_dpad * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_e);
    if (e != cudaSuccess) return e;
    k_mlp_eval<<<p.n_rows, kMlpN / 2, smem_e, st>>>(desc, p.row_exec, rows, p.x, p.y, f_out);
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
