// k_gemm32.cu -- k_rot_simt: the rotation GEMM and objective on the CUDA
// cores in FP32, for the executors an FP32 context puts on the per-generation
// pipeline (every one with D_pad > 256, and those at or above the FP32
// width).  It takes the place of k_rot_tc in the tensor-core pipeline
// (prologue, trial, GEMM + objective, selection, ties).
//
// One CTA (256 threads) per 64-row tile of an executor.  The CTA walks the
// columns of Z in chunks of SN = 256 (64 or 128 when no executor on the path
// is wider); for each chunk it streams K in chunks of 16 through two
// shared-memory buffers: while the current chunk is multiplied, R^T [16][SN]
// of the next one arrives by cp.async and its (u - o)^T [16][64] values
// (formed from the trial rows) wait in registers.  Every thread accumulates
// SN / 64 4x4 blocks of Z (rows 4 tx.., columns 4 (ty0 + 16 j)..) in
// registers.  k ascends in every fma
// chain, so z is bit-identical to the other FP32 rotations.  The chunk of Z
// then goes to shared memory and four lanes per row push it, in column order,
// into the objective's running state (group_obj_push), which carries across
// the chunks; the last chunk gives f.
#include "block.cuh"
#include "group_obj.cuh"
#include "internal.h"

namespace metade {

namespace {
constexpr int kSM = 64;         // rows per tile
constexpr int kSK = 16;         // K per stage
constexpr int kSAP = kSM + 4;   // row length of the (u - o)^T stage

// 16-byte cp.async; src_bytes 0 fills the destination with zeros
__device__ __forceinline__ void cpa16(float* dst, const float* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cpa_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int OBJ>
__device__ __forceinline__ void push_chunk(GroupObj& g, const float* zr, int col0, int ncol, int s, int dim) {
    for (int r0 = 0; r0 < ncol; r0 += 4) group_obj_push<4, OBJ>(OBJ, g, zr[r0 + s], col0 + r0, s, dim);
}
}  // namespace

// SN columns of Z per chunk (64, 128 or 256: the narrowest that covers the widest executor, so
// narrow executors do not compute columns past D); the chunk's row length in shared memory is SN + 4.
template <int SN>
__global__ void __launch_bounds__(256, 2) k_rot_simt(const InstDesc* __restrict__ desc, const int* __restrict__ tiles,
                                                     const float* __restrict__ rows, const float* __restrict__ shift,
                                                     const float* __restrict__ rotT, float* f_out) {
    constexpr int kSN = SN, kSZP = SN + 4, kJ = SN / 64;  // 4x4 column blocks per thread
    extern __shared__ __align__(16) float sm[];
    float* As = sm;                        // 2 x [kSK][kSAP]
    float* Bs = As + 2 * kSK * kSAP;       // 2 x [kSK][kSN]
    float* Zs = Bs + 2 * kSK * kSN;        // [kSM][kSZP]
    const int tid = threadIdx.x;
    const int k = tiles[2 * blockIdx.x], m0 = tiles[2 * blockIdx.x + 1];
    const InstDesc d = desc[k];
    const int dim = d.dim, dp = d.dpad, nv = min(kSM, d.np - m0);
    const float* X = rows + d.pop_off + (long long)m0 * dp;
    const float* o = shift + d.shift_off;
    const float* RT = rotT + d.rot_off;
    const int tx = tid & 15, ty0 = tid >> 4;    // GEMM blocks
    const int orow = tid >> 2, os = tid & 3;    // objective: four lanes per row
    const int nks = (dim + kSK - 1) / kSK;      // K chunks per column chunk
    // this thread's four (u - o) elements of a K chunk: e = tid + 256 q, row t = e / 16, k = e % 16
    auto load_a = [&](int k0, float (&v)[4]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q, t = e / kSK, kk = e - t * kSK;
            v[q] = (t < nv && k0 + kk < dim) ? X[(long long)t * dp + k0 + kk] - o[k0 + kk] : 0.f;
        }
    };
    auto store_a = [&](float* dst, const float (&v)[4]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q, t = e / kSK, kk = e - t * kSK;
            dst[kk * kSAP + t] = v[q];
        }
    };
    auto issue_b = [&](float* dst, int k0, int col0) {
#pragma unroll
        for (int q = 0; q < kJ; ++q) {
            const int e = tid + 256 * q, kk = e / (kSN / 4), c4 = e - kk * (kSN / 4), col = col0 + 4 * c4;
            const bool in = k0 + kk < dim && col < dp;
            cpa16(dst + kk * kSN + 4 * c4, in ? RT + (long long)(k0 + kk) * dp + col : RT, in ? 16 : 0);
        }
        cpa_commit();
    };
    GroupObj g;
    for (int col0 = 0; col0 < dim; col0 += kSN) {
        float acc[kJ][4][4];
#pragma unroll
        for (int j = 0; j < kJ; ++j)
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[j][p][q] = 0.f;
        {
            float v[4];
            load_a(0, v);
            store_a(As, v);
            issue_b(Bs, 0, col0);
            cpa_wait_all();
            __syncthreads();
        }
        for (int it = 0; it < nks; ++it) {
            const int cur = it & 1, k0 = it * kSK, kn = min(kSK, dim - k0);
            const bool more = it + 1 < nks;
            float nxt[4];
            if (more) {
                issue_b(Bs + (cur ^ 1) * kSK * kSN, k0 + kSK, col0);
                load_a(k0 + kSK, nxt);
            }
            const float* Ac = As + cur * kSK * kSAP;
            const float* Bc = Bs + cur * kSK * kSN;
            for (int kk = 0; kk < kn; ++kk) {
                const float4 av = *reinterpret_cast<const float4*>(Ac + kk * kSAP + 4 * tx);
                const float ar[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
                for (int j = 0; j < kJ; ++j) {
                    const float4 rv = *reinterpret_cast<const float4*>(Bc + kk * kSN + 4 * (ty0 + 16 * j));
                    const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[j][p][q] = fmaf(rr[q], ar[p], acc[j][p][q]);
                }
            }
            if (more) {
                store_a(As + (cur ^ 1) * kSK * kSAP, nxt);
                cpa_wait_all();
            }
            __syncthreads();  // the next chunk is in place; this one is free for the chunk after
        }
#pragma unroll
        for (int j = 0; j < kJ; ++j)
#pragma unroll
            for (int p = 0; p < 4; ++p)
                *reinterpret_cast<float4*>(Zs + (4 * tx + p) * kSZP + 4 * (ty0 + 16 * j)) =
                    make_float4(acc[j][p][0], acc[j][p][1], acc[j][p][2], acc[j][p][3]);
        __syncthreads();
        const int ncol = min(kSN, dim - col0);
        const float* zr = Zs + orow * kSZP;
        switch (d.obj) {  // one dispatch per chunk; every lane of the CTA takes part (shuffles)
        case kSphere: push_chunk<kSphere>(g, zr, col0, ncol, os, dim); break;
        case kRosenbrock: push_chunk<kRosenbrock>(g, zr, col0, ncol, os, dim); break;
        case kRastrigin: push_chunk<kRastrigin>(g, zr, col0, ncol, os, dim); break;
        case kGriewank: push_chunk<kGriewank>(g, zr, col0, ncol, os, dim); break;
        case kAckley: push_chunk<kAckley>(g, zr, col0, ncol, os, dim); break;
        default: push_chunk<kSchwefel12>(g, zr, col0, ncol, os, dim); break;
        }
        __syncthreads();
    }
    const float f = group_obj_finish<4>(d.obj, g, dim);
    if (os == 0 && orow < nv) f_out[d.fit_off + m0 + orow] = nan_to_inf(f);
}

int simt_sn(int max_dpad) { return max_dpad <= 64 ? 64 : max_dpad <= 128 ? 128 : 256; }

size_t rot_simt_smem(int max_dpad) {
    const int sn = simt_sn(max_dpad);
    return (size_t)(2 * kSK * kSAP + 2 * kSK * sn + kSM * (sn + 4)) * sizeof(float);
}

template <int SN>
static cudaError_t launch_rot_simt_sn(const InstDesc* desc, const int* tiles, int n_tiles, const float* rows,
                                      const float* shift, const float* rotT, float* f_out, size_t smem,
                                      cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_rot_simt<SN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_rot_simt<SN><<<n_tiles, 256, smem, st>>>(desc, tiles, rows, shift, rotT, f_out);
    return cudaGetLastError();
}

cudaError_t launch_rot_simt(const InstDesc* desc, const int* tiles, int n_tiles, const float* rows, const float* shift,
                            const float* rotT, float* f_out, int max_dpad, cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    const size_t smem = rot_simt_smem(max_dpad);
    switch (simt_sn(max_dpad)) {
    case 64: return launch_rot_simt_sn<64>(desc, tiles, n_tiles, rows, shift, rotT, f_out, smem, st);
    case 128: return launch_rot_simt_sn<128>(desc, tiles, n_tiles, rows, shift, rotT, f_out, smem, st);
    default: return launch_rot_simt_sn<256>(desc, tiles, n_tiles, rows, shift, rotT, f_out, smem, st);
    }
}

}  // namespace metade
