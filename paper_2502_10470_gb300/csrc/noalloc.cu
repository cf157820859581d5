// noalloc.cu -- metade_plain_step_noalloc: one plain FP32 generation of a
// single executor that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs where the device heap
// is owned by someone else (a host framework with its own caching allocator
// that forbids outside allocations, a plugin that must not grow the process's
// device footprint, or code issued while the device allocator is unavailable).
// This entry point takes every input and output as caller memory and keeps the
// scratch the plain kernels need (trial rows, trial fitness, the pbest pool)
// in one file-scope device array of fixed size instead of in a context.
//
// The array is part of the library image: every GPU that loads the library
// holds it until the process exits.  All calls share it and it keeps the last
// call's contents; every element a call reads is written earlier in the same
// call, so nothing is cleared.  Two calls that overlap on the GPU (different
// streams, or different host threads on one device) race on it.
//
// Host code must not pass the array's name to a kernel: on the host it is a
// stand-in symbol, not a device address.  The device address is obtained with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made while it is current; that first call should therefore come
// before any stream capture.  The address is cached for the life of the
// process: after cudaDeviceReset (or anything else that destroys the device's
// primary context and unloads the library's device code) the cached address
// is stale, so a process that resets a device must not call this entry point
// on that device again.
#include <cstring>
#include <mutex>

#include "../../include/metade.h"
#include "block.cuh"

using namespace metade;

namespace {

constexpr long long kScratchFloats = 1LL << 20;  // 4 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) float g_noalloc_scratch[kScratchFloats];
__device__ int g_noalloc_status;  // the last call: 0 generation run, 1 skipped (invalid theta)

std::mutex g_mu;
float* g_scratch_dev[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

// z = R d by one warp, lanes own rows; R row-major [dim][dim] (unpadded).
__device__ __forceinline__ void warp_rotate_rowmajor(int dim, const float* R, const float* d, float* z) {
    const int lane = threadIdx.x & 31;
    for (int r = lane; r < dim; r += 32) {
        const float* row = R + (size_t)r * dim;
        float acc = 0.f;
        for (int c = 0; c < dim; ++c) acc = fmaf(row[c], d[c], acc);
        z[r] = acc;
    }
}

__device__ __forceinline__ void warp_rotate_pair_rowmajor(int dim, const float* R, const float* x, const float* u,
                                                          const float* o, float* z, float* dz) {
    const int lane = threadIdx.x & 31;
    for (int r = lane; r < dim; r += 32) {
        const float* row = R + (size_t)r * dim;
        float az = 0.f, ad = 0.f;
        for (int c = 0; c < dim; ++c) {
            az = fmaf(row[c], x[c] - o[c], az);
            ad = fmaf(row[c], u[c] - x[c], ad);
        }
        z[r] = az;
        dz[r] = ad;
    }
}

struct NaArgs {
    InstDesc d;           // executor description (offsets 0)
    float* pop;           // [np][dpad]
    float* fit;           // [np]
    const float* theta;   // [6]
    const float* shift;   // [dim]
    const float* rot;     // [dim][dim] row-major
    Key key;
    uint32_t epoch, gen;
    float lo, hi;
    float* u;             // scratch: trial rows [np][dpad]
    float* fu;            // scratch: trial fitness [np]
    int* topk;            // scratch: pbest pool [np]
};

__global__ void k_na_prologue(NaArgs a) {
    const Strat s = load_strat(a.theta, a.d.np);
    if (threadIdx.x == 0) g_noalloc_status = s.ok ? 0 : 1;
    if (!s.ok) return;
    block_topk_staged(a.fit, a.d.np, a.d.kp, a.topk);
}

__global__ void __launch_bounds__(256) k_na_trial(NaArgs a) {
    extern __shared__ __align__(16) float sm[];
    const InstDesc& d = a.d;
    const Strat s = load_strat(a.theta, d.np);
    if (!s.ok) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= d.np) return;
    float* db = sm + (size_t)warp * 2 * d.dpad;
    float* zb = db + d.dpad;
    const Ctr c = make_ctr(a.key, (uint32_t)d.stream, a.gen, (uint32_t)i, a.epoch);
    Indiv v;
    indiv_setup(s, c, i, d.np, d.dim, d.kp, a.topk, a.topk[0], v);
    const int L = s.cs == 2 ? exp_length(c, d.dim, s.cri) : 0;
    warp_trial(s, c, v, i, d.dim, L, a.pop, d.dpad, a.shift, a.lo, a.hi, a.u + (long long)i * d.dpad, db);
    __syncwarp();
    warp_rotate_rowmajor(d.dim, a.rot, db, zb);
    __syncwarp();
    const float f = warp_objective<float>(d.obj, d.dim, zb);
    if (lane == 0) a.fu[i] = nan_to_inf(f);
}

__global__ void __launch_bounds__(256) k_na_select(NaArgs a) {
    extern __shared__ __align__(16) float sm[];
    const InstDesc& d = a.d;
    const Strat s = load_strat(a.theta, d.np);
    if (!s.ok) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= d.np) return;
    float* X = a.pop + (long long)i * d.dpad;
    const float* U = a.u + (long long)i * d.dpad;
    float fn = a.fu[i];
    const float fx = a.fit[i];
    bool take;
    bool tie = near_tie(fn, fx, tie_band(d.dim));
    if (tie) {
        bool diff = false;
        for (int j = lane; j < d.dim; j += 32) diff = diff || (U[j] != X[j]);
        if (!__any_sync(kFull, diff)) tie = false, fn = fx;  // trial == target
    }
    if (tie) {
        float* zb = sm + (size_t)warp * 2 * d.dpad;
        warp_rotate_pair_rowmajor(d.dim, a.rot, X, U, a.shift, zb, zb + d.dpad);
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
        if (lane == 0) a.fit[i] = fn;
    }
}

}  // namespace

extern "C" METADE_API metade_status metade_plain_step_noalloc(float* pop, float* fit, const float* theta,
                                                              const float* shift, const float* rot, int32_t np,
                                                              int32_t dim, int32_t obj, float lo, float hi,
                                                              uint64_t seed, uint32_t stream_id, uint32_t epoch,
                                                              uint32_t gen, int32_t p_best_pct, void* stream) {
    if (!pop || !fit || !theta || !shift || !rot) return METADE_EINVAL;
    if (reinterpret_cast<uintptr_t>(pop) & 15) return METADE_EINVAL;  // rows are read and written as float4
    if (np < 4 || np > 1024 || dim < 1 || dim > 1536 || obj < 0 || obj > 5 || epoch > 0xFFFFu) return METADE_EINVAL;
    if (!(lo < hi) || p_best_pct < 0 || p_best_pct > 100) return METADE_EINVAL;
    const int dpad = (dim + 3) & ~3;
    const long long u_floats = (long long)np * dpad;
    const long long fu_off = (u_floats + 63) & ~63LL;
    const long long topk_off = (fu_off + np + 63) & ~63LL;
    if (topk_off + np > kScratchFloats) return METADE_EINVAL;  // beyond the fixed scratch (4 MiB)
    float* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return METADE_ECUDA;
    const int pct = p_best_pct == 0 ? 10 : p_best_pct;

    NaArgs a;
    std::memset(&a.d, 0, sizeof(a.d));
    a.d.np = np;
    a.d.dim = dim;
    a.d.dpad = dpad;
    a.d.obj = obj;
    a.d.stream = (int)stream_id;
    a.d.kp = (np * pct + 99) / 100 < 1 ? 1 : (np * pct + 99) / 100;
    a.pop = pop;
    a.fit = fit;
    a.theta = theta;
    a.shift = shift;
    a.rot = rot;
    a.key = make_key(seed, kTagInner);
    a.epoch = epoch;
    a.gen = gen;
    a.lo = lo;
    a.hi = hi;
    a.u = scratch;
    a.fu = scratch + fu_off;
    a.topk = reinterpret_cast<int*>(scratch + topk_off);

    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (np + 7) / 8;
    const size_t smem = (size_t)8 * 2 * dpad * sizeof(float);
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(k_na_trial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ||
            cudaFuncSetAttribute(k_na_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
            return METADE_ECUDA;
    }
    // each launch is checked with cudaPeekAtLastError, which leaves the error
    // state of other code untouched (cudaGetLastError would clear it)
    k_na_prologue<<<1, 256, 0, st>>>(a);
    if (cudaPeekAtLastError() != cudaSuccess) return METADE_ECUDA;
    k_na_trial<<<blocks, 256, smem, st>>>(a);
    if (cudaPeekAtLastError() != cudaSuccess) return METADE_ECUDA;
    k_na_select<<<blocks, 256, smem, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? METADE_OK : METADE_ECUDA;
}

extern "C" METADE_API metade_status metade_plain_step_noalloc_status(int32_t* status) {
    if (!status) return METADE_EINVAL;
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_noalloc_status, sizeof(int)) != cudaSuccess) return METADE_ECUDA;
    *status = v;
    return METADE_OK;
}
