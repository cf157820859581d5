// block.cuh -- block- and warp-level helpers shared by the step kernels:
// best (argmin, lowest index on ties) and the pbest pool (top k_p by stored
// fitness, Sec. II-A), warp-parallel objectives over a z vector held in
// shared memory, and the warp-per-individual trial construction.
#pragma once
#include "device.cuh"

namespace metade {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ bool better(float fa, int ia, float fb, int ib) {
    return fa < fb || (fa == fb && ia < ib);
}

// argmin of f[0..np) with the lowest index on ties; every thread receives it.
// `red` is shared scratch of >= 64 words.  Contains __syncthreads.
__device__ __forceinline__ int block_argmin(const float* f, int np, int* red) {
    float bv = INFINITY;
    int bi = 0x7FFFFFFF;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const float v = f[i];
        if (better(v, i, bv, bi)) { bv = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(kFull, bv, o);
        const int oi = __shfl_xor_sync(kFull, bi, o);
        if (better(ov, oi, bv, bi)) { bv = ov; bi = oi; }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    float* rv = reinterpret_cast<float*>(red);
    int* ri = red + 32;
    __syncthreads();
    if (lane == 0) { rv[warp] = bv; ri[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
        bv = lane < nw ? rv[lane] : INFINITY;
        bi = lane < nw ? ri[lane] : 0x7FFFFFFF;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(kFull, bv, o);
            const int oi = __shfl_xor_sync(kFull, bi, o);
            if (better(ov, oi, bv, bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) ri[0] = (bi == 0x7FFFFFFF) ? 0 : bi;
    }
    __syncthreads();
    const int r = ri[0];
    __syncthreads();
    return r;
}

// The pbest pool: topk[rank] = i for the k_p best individuals by (f, index).
// Each individual counts how many are better (rank); a warp stops scanning
// once every lane knows its rank is >= k_p.  Contains no barrier; callers
// __syncthreads before reading topk.
__device__ __forceinline__ void block_topk(const float* f, int np, int kp, int* topk) {
    for (int base = 0; base < np; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const bool active = i < np;
        const float fi = active ? f[i] : 0.0f;
        int rank = 0;
        bool done = !active;
        for (int j0 = 0; j0 < np; j0 += 32) {
            if (__all_sync(kFull, done)) break;
            if (j0 + 32 <= np) {  // a whole block of 32: the loads issue back to back
#pragma unroll 8
                for (int jj = 0; jj < 32; ++jj) rank += better(f[j0 + jj], j0 + jj, fi, i) ? 1 : 0;
            } else {
                for (int j = j0; j < np; ++j) rank += better(f[j], j, fi, i) ? 1 : 0;
            }
            done = done || rank >= kp;
        }
        if (active && rank < kp) topk[rank] = i;
    }
}

// block_topk of fitness in global memory, on a copy in shared memory: each
// thread's rank scan reads the whole array, which from global memory is bound
// by its latency.  np <= kTopkStage (larger arrays are scanned where they
// are).  Contains __syncthreads; callers __syncthreads before reading topk.
constexpr int kTopkStage = 1024;
__device__ __forceinline__ void block_topk_staged(const float* f, int np, int kp, int* topk) {
    __shared__ float sf[kTopkStage];
    if (np > kTopkStage) {
        block_topk(f, np, kp, topk);
        return;
    }
    for (int i = threadIdx.x; i < np; i += blockDim.x) sf[i] = f[i];
    __syncthreads();
    block_topk(sf, np, kp, topk);
}

// ------------------------------------------------------ warp reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_prod(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(kFull, v, o);
    return v;
}

// Objective of z[0..dim) (shared memory) computed by one warp; every lane
// returns the value.  Same stable forms as the streaming accumulator.
template <typename T>
__device__ __forceinline__ T warp_objective(int obj, int dim, const T* z) {
    const int lane = threadIdx.x & 31;
    T s0 = T(0), s1 = T(0), prod = T(1);
    bool pos = true;
    if (obj == kSchwefel12) {
        T carry = T(0);
        for (int j0 = 0; j0 < dim; j0 += 32) {
            const int j = j0 + lane;
            T x = j < dim ? z[j] : T(0);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const T y = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += y;
            }
            const T p = carry + x;
            if (j < dim) s0 += p * p;
            carry += __shfl_sync(kFull, x, 31);
        }
        return warp_sum(s0);
    }
    for (int j = lane; j < dim; j += 32) {
        const T zj = z[j];
        switch (obj) {
        case kSphere: s0 += zj * zj; break;
        case kRosenbrock:
            if (j + 1 < dim) {
                const T t = z[j + 1] - zj * (zj + T(2));
                s0 += T(100) * t * t + zj * zj;
            }
            break;
        case kRastrigin: {
            const T s = sinpi_t<T>(zj);
            s0 += zj * zj + T(20) * s * s;
            break;
        }
        case kGriewank: {
            s0 += zj * zj;
            const T arg = zj / sqrt(T(j + 1));
            const T h = sin(arg * T(0.5));
            s1 += log1p(T(-2) * h * h);
            const T c = cos(arg);
            pos = pos && (c > T(0));
            prod *= c;
            break;
        }
        case kAckley: {
            s0 += zj * zj;
            const T s = sinpi_t<T>(zj);
            s1 += s * s;
            break;
        }
        }
    }
    s0 = warp_sum(s0);
    if (obj == kGriewank) {
        s1 = warp_sum(s1);
        prod = warp_prod(prod);
        pos = __all_sync(kFull, pos);
        return s0 / T(4000) + (pos ? -expm1(s1) : (T(1) - prod));
    }
    if (obj == kAckley) {
        s1 = warp_sum(s1);
        const T r = sqrt(s0 / T(dim));
        return T(-20) * expm1(T(-0.2) * r) - T(2.71828182845904523536) * expm1(T(-2) * s1 / T(dim));
    }
    return s0;
}

// z = R d by one warp, lanes own rows.  RT: transposed rotation [dim][ldr]
// (RT[c * ldr + r] = R[r][c]); d: shared, dim values (pad to a multiple of 4,
// zero-filled).  Writes z[r] (shared).
template <typename T>
__device__ __forceinline__ void warp_rotate(int dim, const float* RT, int ldr, const float* d, T* z) {
    const int lane = threadIdx.x & 31;
    for (int r0 = 0; r0 < dim; r0 += 32) {
        const int r = r0 + lane;
        const bool act = r < dim;
        T acc = T(0);
        int c = 0;
        for (; c + 4 <= dim; c += 4) {
            const float4 dv = *reinterpret_cast<const float4*>(d + c);
            if (act) {
                acc = fma(T(RT[(size_t)(c + 0) * ldr + r]), T(dv.x), acc);
                acc = fma(T(RT[(size_t)(c + 1) * ldr + r]), T(dv.y), acc);
                acc = fma(T(RT[(size_t)(c + 2) * ldr + r]), T(dv.z), acc);
                acc = fma(T(RT[(size_t)(c + 3) * ldr + r]), T(dv.w), acc);
            }
        }
        for (; c < dim; ++c)
            if (act) acc = fma(T(RT[(size_t)c * ldr + r]), T(d[c]), acc);
        if (act) z[r] = acc;
    }
}

// FP64 evaluation of one float32 point by a warp (selection ties, FP64
// evaluation).  dbuf/zbuf: shared double scratch of >= dim entries.
__device__ __forceinline__ double warp_eval64(int obj, int dim, const float* x, const float* o, const float* RT,
                                              int ldr, double* dbuf, double* zbuf) {
    const int lane = threadIdx.x & 31;
    for (int j = lane; j < dim; j += 32) dbuf[j] = (double)x[j] - (double)o[j];
    __syncwarp();
    for (int r0 = 0; r0 < dim; r0 += 32) {
        const int r = r0 + lane;
        if (r < dim) {
            double acc = 0.0;
            for (int c = 0; c < dim; ++c) acc = fma((double)RT[(size_t)c * ldr + r], dbuf[c], acc);
            zbuf[r] = acc;
        }
    }
    __syncwarp();
    const double f = warp_objective<double>(obj, dim, zbuf);
    __syncwarp();
    return f;
}

// z = R (x - o) and dz = R (u - x) by one warp, lanes own rows (tie decisions).
__device__ __forceinline__ void warp_rotate_pair(int dim, const float* RT, int ldr, const float* x, const float* u,
                                                 const float* o, float* z, float* dz) {
    const int lane = threadIdx.x & 31;
    for (int r0 = 0; r0 < dim; r0 += 32) {
        const int r = r0 + lane;
        float az = 0.f, ad = 0.f;
        if (r < dim)
            for (int c = 0; c < dim; ++c) {
                const float rt = RT[(size_t)c * ldr + r];
                az = fmaf(rt, x[c] - o[c], az);
                ad = fmaf(rt, u[c] - x[c], ad);
            }
        if (r < dim) {
            z[r] = az;
            dz[r] = ad;
        }
    }
}

// z = R (x - o) and dz = R (u - x) by one warp with the two operand vectors
// staged in shared memory first (coalesced row reads), then one pass over R^T
// for both (each coalesced R^T load feeds two fma chains; the operands are
// broadcast reads).  buf: 4 * ldb floats of shared scratch; z and dz are left
// in buf + 2 ldb and buf + 3 ldb.  Same fma chain per row as warp_rotate.
__device__ __forceinline__ void warp_rotate_pair_staged(int dim, const float* RT, int ldr, const float* x,
                                                        const float* u, const float* o, float* buf, int ldb) {
    const int lane = threadIdx.x & 31;
    float* dx = buf;
    float* dl = buf + ldb;
    float* z = buf + 2 * ldb;
    float* dz = buf + 3 * ldb;
    const int d4 = (dim + 3) & ~3;
    for (int j = lane; j < d4; j += 32) {
        const bool in = j < dim;
        const float xv = in ? x[j] : 0.f;
        dx[j] = in ? xv - o[j] : 0.f;
        dl[j] = in ? u[j] - xv : 0.f;
    }
    __syncwarp();
    for (int r0 = 0; r0 < dim; r0 += 32) {
        const int r = r0 + lane;
        const bool act = r < dim;
        float az = 0.f, ad = 0.f;
        for (int c = 0; c < d4; c += 4) {
            const float4 xv = *reinterpret_cast<const float4*>(dx + c);
            const float4 lv = *reinterpret_cast<const float4*>(dl + c);
            if (act) {
                const float xs[4] = {xv.x, xv.y, xv.z, xv.w}, ls[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (c + q < dim) {
                        const float rt = RT[(size_t)(c + q) * ldr + r];
                        az = fmaf(rt, xs[q], az);
                        ad = fmaf(rt, ls[q], ad);
                    }
                }
            }
        }
        if (act) {
            z[r] = az;
            dz[r] = ad;
        }
    }
    __syncwarp();
}

// f(u) - f(x) from z, dz (shared) by one warp; same difference forms as the
// streaming DiffAcc.  Every lane returns the value.
__device__ __forceinline__ float warp_diff(int obj, int dim, const float* z, const float* dz) {
    const int lane = threadIdx.x & 31;
    if (obj == kSchwefel12) {
        float cz = 0.f, cd = 0.f, s = 0.f;
        for (int j0 = 0; j0 < dim; j0 += 32) {
            const int j = j0 + lane;
            float x = j < dim ? z[j] : 0.f, y = j < dim ? dz[j] : 0.f;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const float xs = __shfl_up_sync(kFull, x, o), ys = __shfl_up_sync(kFull, y, o);
                if (lane >= o) {
                    x += xs;
                    y += ys;
                }
            }
            const float p = cz + x, dp = cd + y;
            if (j < dim) s += dp * (2.f * p + dp);
            cz += __shfl_sync(kFull, x, 31);
            cd += __shfl_sync(kFull, y, 31);
        }
        return warp_sum(s);
    }
    float d0 = 0.f, d1 = 0.f, x0 = 0.f, x1 = 0.f, lr = 0.f, px = 1.f;
    for (int j = lane; j < dim; j += 32) {
        const float zj = z[j], dj = dz[j];
        switch (obj) {
        case kSphere: d0 += dj * (2.f * zj + dj); break;
        case kRosenbrock:
            if (j + 1 < dim) {
                const float t = z[j + 1] - zj * (zj + 2.f);
                const float dt = dz[j + 1] - dj * (2.f * zj + 2.f + dj);
                d0 += 100.f * dt * (2.f * t + dt) + dj * (2.f * zj + dj);
            }
            break;
        case kRastrigin: d0 += dj * (2.f * zj + dj) + 20.f * sin_pi(2.f * zj + dj) * sin_pi(dj); break;
        case kGriewank: {
            // per lane: (A, B) with A = prod c, B = prod c' - prod c over its
            // coordinates; combined across lanes in index order below
            d0 += dj * (2.f * zj + dj);
            const float inv = rsqrtf((float)(j + 1));
            const float ang = zj * inv, da = dj * inv;
            float c;
            const float dc = cos_step(ang, 0.5f * da, c);
            lr = (c + dc) * lr + dc * px;
            px *= c;
            break;
        }
        case kAckley: {
            x0 += zj * zj;
            d0 += dj * (2.f * zj + dj);
            x1 += sin2pi(zj);
            d1 += sin_pi(2.f * zj + dj) * sin_pi(dj);
            break;
        }
        }
    }
    d0 = warp_sum(d0);
    if (obj == kGriewank) {
        // Each lane holds, for its coordinates j = lane, lane+32, ... (in
        // increasing order), the product A = prod c and B = prod c' - prod c.
        // Segments compose as (A1, B1) then (A2, B2): A = A1 A2,
        // B = (A1 + B1) B2 + B1 A2.  The lanes' coordinate sets interleave,
        // but a product does not depend on the order of its factors, so the
        // lane values compose in any order.
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float A2 = __shfl_xor_sync(kFull, px, o), B2 = __shfl_xor_sync(kFull, lr, o);
            const float A1 = px, B1 = lr;
            px = A1 * A2;
            lr = (A1 + B1) * B2 + B1 * A2;
        }
        return d0 / 4000.f - lr;
    }
    if (obj == kAckley) {
        d1 = warp_sum(d1);
        x0 = warp_sum(x0);
        x1 = warp_sum(x1);
        const float rx = sqrtf(x0 / dim), ru = sqrtf(fmaxf(x0 + d0, 0.f) / dim);
        const float dr = (ru + rx > 0.f) ? (d0 / dim) / (ru + rx) : 0.f;
        return -20.f * expf(-0.2f * rx) * expm1f(-0.2f * dr) -
               2.71828182845904523536f * expf(-2.f * x1 / dim) * expm1f(-2.f * d1 / dim);
    }
    return d0;
}

// One 4-coordinate chunk j4..j4+3 of a trial: mutation from the loaded base
// rows (a = x_bl, b = x_br, x = x_i) and the summed difference vectors
// (sum = sum_q x_plus - x_minus, added in q order), then crossover (binomial
// words w, exponential start/length, arithmetic K), clip to [lo, hi].  u
// gets the trial coordinates (0 past dim), d the shifted ones u - o (0 past
// dim).  Every trial kernel goes through this one function, so trials are
// bit-identical whichever kernel builds them.
__device__ __forceinline__ void trial_chunk(const Strat& s, float K, int jrand, int nstart, int L, int dim, int j4,
                                            const float4& a, const float4& b, const float4& x, const float4& sum,
                                            const uint4& w, const float* o, float lo, float hi, float (&uo)[4],
                                            float (&dd)[4]) {
    const float F = s.F;
    const bool dir = s.bl != s.br;
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
    const float xv[4] = {x.x, x.y, x.z, x.w}, sv[4] = {sum.x, sum.y, sum.z, sum.w};
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
                take = ((word_of(w, q) >> 8) < s.cri) || (j == jrand);
            } else {
                int off = j - nstart;
                if (off < 0) off += dim;
                take = off < L;
            }
            u = take ? vj : xv[q];
        }
        u = fminf(fmaxf(u, lo), hi);
        if (j >= dim) u = 0.0f;
        uo[q] = u;
        dd[q] = (j < dim) ? (u - o[j]) : 0.0f;
    }
}

// Trial vector of individual i built by one warp, four coordinates per lane
// and step: mutation, crossover and clip (trial_chunk).  X: generation-start
// rows (stride ldx); U: trial row out (global or shared, 16-byte aligned);
// u - o of the four coordinates (zero past dim) is handed to sink(j4, dd).
template <typename Sink>
__device__ __forceinline__ void warp_trial_to(const Strat& s, const Ctr& c, const Indiv& v, int i, int dim, int L,
                                              const float* X, long long ldx, const float* o, float lo, float hi,
                                              float* U, Sink&& sink) {
    const int lane = threadIdx.x & 31;
    const float K = (float)v.kraw * (1.0f / 16777216.0f);
    const float* xl = X + (long long)v.ibl * ldx;
    const float* xr = X + (long long)v.ibr * ldx;
    const float* xi = X + (long long)i * ldx;
    for (int j4 = lane * 4; j4 < dim; j4 += 128) {
        const float4 a = *reinterpret_cast<const float4*>(xl + j4);
        const float4 b = *reinterpret_cast<const float4*>(xr + j4);
        const float4 x = *reinterpret_cast<const float4*>(xi + j4);
        float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q = 0; q < s.dn; ++q) {
            const float4 p = *reinterpret_cast<const float4*>(X + (long long)diff_plus(v, s.a, q) * ldx + j4);
            const float4 m = *reinterpret_cast<const float4*>(X + (long long)diff_minus(v, s.a, q) * ldx + j4);
            sum.x += p.x - m.x; sum.y += p.y - m.y; sum.z += p.z - m.z; sum.w += p.w - m.w;
        }
        const uint4 w = (s.cs == 1) ? c.slot(4 + (uint32_t)(j4 >> 2)) : make_uint4(0, 0, 0, 0);
        float uo[4], dd[4];
        trial_chunk(s, K, v.jrand, v.nstart, L, dim, j4, a, b, x, sum, w, o, lo, hi, uo, dd);
        *reinterpret_cast<float4*>(U + j4) = make_float4(uo[0], uo[1], uo[2], uo[3]);
        sink(j4, dd);
    }
}

// warp_trial_to with u - o stored to dbuf (shared, dim rounded up to 4); the
// warp must __syncwarp before reading dbuf
__device__ __forceinline__ void warp_trial(const Strat& s, const Ctr& c, const Indiv& v, int i, int dim, int L,
                                           const float* X, long long ldx, const float* o, float lo, float hi,
                                           float* U, float* dbuf) {
    warp_trial_to(s, c, v, i, dim, L, X, ldx, o, lo, hi, U, [&](int j4, const float (&dd)[4]) {
        *reinterpret_cast<float4*>(dbuf + j4) = make_float4(dd[0], dd[1], dd[2], dd[3]);
    });
}

}  // namespace metade
