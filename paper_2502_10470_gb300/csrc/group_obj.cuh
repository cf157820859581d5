// group_obj.cuh -- objective of one individual evaluated by a group of S
// consecutive lanes of a warp (S = 2, 4, 8) that receive its rotated rows in
// blocks of S: in block r0 lane s holds z of row r0 + s.  Every lane of the
// warp must call the push and finish functions (they shuffle with the full
// mask).  The FP32 forms are those of the per-thread objective (device.cuh):
// Griewank as the telescoping pair (P = prod c_j, Q = 1 - P) composed across
// lanes, Rosenbrock pairing each row with its successor across lanes and
// blocks, Schwefel 1.2 as a group scan plus a carry.
#pragma once
#include "device.cuh"

namespace metade {

template <int S>
__device__ __forceinline__ float gsum(float v) {
#pragma unroll
    for (int o = 1; o < S; o <<= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <int S>
__device__ __forceinline__ int gmin(int v) {
#pragma unroll
    for (int o = 1; o < S; o <<= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

template <int S>
__device__ __forceinline__ bool gany(bool v) {
    unsigned x = v ? 1u : 0u;
#pragma unroll
    for (int o = 1; o < S; o <<= 1) x |= __shfl_xor_sync(kFull, x, o);
    return x != 0;
}

struct GroupObj {
    float s0 = 0.f, s1 = 0.f;        // sums
    float P = 1.f, Q = 0.f;          // Griewank product pair: P = prod c, Q = 1 - P
    float pend = 0.f;                // Rosenbrock: this lane's last row waiting for its successor
    bool has_pend = false;
    float carry = 0.f;               // Schwefel: prefix of all previous blocks
};

// Row block r0: this lane contributes z of row r0 + s (ignored past dim).
// OBJ < 0: the objective is the runtime value obj.
template <int S, int OBJ = -1>
__device__ __forceinline__ void group_obj_push(int obj, GroupObj& acc, float z, int r0, int s, int dim) {
    const int r = r0 + s;
    const bool valid = r < dim;
    if (OBJ >= 0) obj = OBJ;
    switch (obj) {
    case kSphere:
        if (valid) acc.s0 = fmaf(z, z, acc.s0);
        break;
    case kRastrigin:
        if (valid) acc.s0 += z * z + 20.f * sin2pi(z);
        break;
    case kAckley:
        if (valid) {
            acc.s0 = fmaf(z, z, acc.s0);
            acc.s1 += sin2pi(z);
        }
        break;
    case kGriewank:
        if (valid) {
            acc.s0 = fmaf(z, z, acc.s0);
            const float wq = 2.f * sin2pi(z * (rsqrtf((float)(r + 1)) * kInv2Pi));  // 2 sin^2(z / (2 sqrt j))
            acc.Q = fmaf(acc.P, wq, acc.Q);
            acc.P *= 1.f - wq;
        }
        break;
    case kRosenbrock: {
        // term of row j = r uses z_{j+1}: the next lane's z, or the next block's lane 0
        const float nxt = __shfl_down_sync(kFull, z, 1, S);
        const float first_next = __shfl_sync(kFull, z, 0, S);  // lane 0 of this block
        // the previous block's last row (held by lane S-1) pairs with this block's first row
        if (acc.has_pend && r0 < dim) {
            const float zj = acc.pend;
            const float t = first_next - zj * (zj + 2.f);
            acc.s0 += 100.f * t * t + zj * zj;
            acc.has_pend = false;
        }
        if (valid && r + 1 < dim) {
            if (s < S - 1) {
                const float t = nxt - z * (z + 2.f);
                acc.s0 += 100.f * t * t + z * z;
            } else {
                acc.pend = z;
                acc.has_pend = true;
            }
        }
        break;
    }
    default: {  // Schwefel 1.2: group inclusive scan of the block plus the carry
        float x = valid ? z : 0.f;
#pragma unroll
        for (int off = 1; off < S; off <<= 1) {
            const float y = __shfl_up_sync(kFull, x, off, S);
            if (s >= off) x += y;
        }
        const float pfx = acc.carry + x;
        if (valid) acc.s0 = fmaf(pfx, pfx, acc.s0);
        acc.carry += __shfl_sync(kFull, x, S - 1, S);
        break;
    }
    }
}

// f of the individual from the lanes' partial state; every lane gets it.
template <int S>
__device__ __forceinline__ float group_obj_finish(int obj, GroupObj& acc, int dim) {
    if (obj == kGriewank) {
#pragma unroll
        for (int off = 1; off < S; off <<= 1) {
            const float P2 = __shfl_xor_sync(kFull, acc.P, off), Q2 = __shfl_xor_sync(kFull, acc.Q, off);
            acc.Q = acc.Q + acc.P * Q2;
            acc.P *= P2;
        }
        return gsum<S>(acc.s0) * (1.f / 4000.f) + acc.Q;
    } else if (obj == kAckley) {
        const float s0 = gsum<S>(acc.s0), s1 = gsum<S>(acc.s1);
        return -20.f * expm1f(-0.2f * sqrtf(s0 / dim)) -
               2.71828182845904523536f * expm1f(-2.f * s1 / dim);
    } else {
        return gsum<S>(acc.s0);
    }
}

// Difference f(u) - f(x) of one individual by a group of S lanes from the
// rows of z = R (x - o) and dz = R (u - x), in blocks of S rows like the
// objective above.  The forms avoid the cancellation of f(u) - f(x):
//   sum of squares   dz (2 z + dz)
//   Rastrigin        adds 20 sin(pi (2 z + dz)) sin(pi dz)
//   Rosenbrock       t = z_{j+1} - z_j (z_j + 2) changes by
//                    dt = dz_{j+1} - dz_j (2 z_j + 2 + dz_j)
//   Griewank         per lane (A, B) = (prod c, prod c' - prod c), composed
//   Ackley           both exponentials as exp(a) expm1(da)
//   Schwefel 1.2     prefix sums p, dp: dp (2 p + dp)
struct GroupDiff {
    float d0 = 0.f, d1 = 0.f, x0 = 0.f, x1 = 0.f, A = 1.f, B = 0.f;
    float pz = 0.f, pdz = 0.f, cz = 0.f, cd = 0.f;
    bool has_pend = false;
};

template <int S, int OBJ = -1>
__device__ __forceinline__ void group_diff_push(int obj, GroupDiff& g, float z, float dz, int r0, int s, int dim) {
    const int r = r0 + s;
    const bool valid = r < dim;
    if (OBJ >= 0) obj = OBJ;
    switch (obj) {
    case kSphere:
        if (valid) g.d0 += dz * (2.f * z + dz);
        break;
    case kRastrigin:
        if (valid) g.d0 += dz * (2.f * z + dz) + 20.f * sin_pi(2.f * z + dz) * sin_pi(dz);
        break;
    case kAckley:
        if (valid) {
            g.x0 = fmaf(z, z, g.x0);
            g.d0 += dz * (2.f * z + dz);
            g.x1 += sin2pi(z);
            g.d1 += sin_pi(2.f * z + dz) * sin_pi(dz);
        }
        break;
    case kGriewank:
        if (valid) {
            g.d0 += dz * (2.f * z + dz);
            const float inv = rsqrtf((float)(r + 1));
            float c;
            const float dc = cos_step(z * inv, 0.5f * dz * inv, c);
            g.B = (c + dc) * g.B + dc * g.A;
            g.A *= c;
        }
        break;
    case kRosenbrock: {
        const float nz = __shfl_down_sync(kFull, z, 1, S), nd = __shfl_down_sync(kFull, dz, 1, S);
        const float fz = __shfl_sync(kFull, z, 0, S), fd = __shfl_sync(kFull, dz, 0, S);
        if (g.has_pend) {  // previous block's last row with this block's first row
            const float t = fz - g.pz * (g.pz + 2.f);
            const float dt = fd - g.pdz * (2.f * g.pz + 2.f + g.pdz);
            g.d0 += 100.f * dt * (2.f * t + dt) + g.pdz * (2.f * g.pz + g.pdz);
            g.has_pend = false;
        }
        if (valid && r + 1 < dim) {
            if (s < S - 1) {
                const float t = nz - z * (z + 2.f);
                const float dt = nd - dz * (2.f * z + 2.f + dz);
                g.d0 += 100.f * dt * (2.f * t + dt) + dz * (2.f * z + dz);
            } else {
                g.pz = z;
                g.pdz = dz;
                g.has_pend = true;
            }
        }
        break;
    }
    default: {  // Schwefel 1.2: prefix sums of z and dz over the rows
        float xs = valid ? z : 0.f, ys = valid ? dz : 0.f;
#pragma unroll
        for (int off = 1; off < S; off <<= 1) {
            const float a2 = __shfl_up_sync(kFull, xs, off, S), b2 = __shfl_up_sync(kFull, ys, off, S);
            if (s >= off) {
                xs += a2;
                ys += b2;
            }
        }
        const float p = g.cz + xs, dp2 = g.cd + ys;
        if (valid) g.d0 += dp2 * (2.f * p + dp2);
        g.cz += __shfl_sync(kFull, xs, S - 1, S);
        g.cd += __shfl_sync(kFull, ys, S - 1, S);
        break;
    }
    }
}

template <int S>
__device__ __forceinline__ float group_diff_finish(int obj, GroupDiff& g, int dim) {
    g.d0 = gsum<S>(g.d0);
    if (obj == kGriewank) {
#pragma unroll
        for (int off = 1; off < S; off <<= 1) {
            const float A2 = __shfl_xor_sync(kFull, g.A, off), B2 = __shfl_xor_sync(kFull, g.B, off);
            g.B = (g.A + g.B) * B2 + g.B * A2;
            g.A *= A2;
        }
        return g.d0 / 4000.f - g.B;
    }
    if (obj == kAckley) {
        g.d1 = gsum<S>(g.d1);
        g.x0 = gsum<S>(g.x0);
        g.x1 = gsum<S>(g.x1);
        const float rx = sqrtf(g.x0 / dim), ru = sqrtf(fmaxf(g.x0 + g.d0, 0.f) / dim);
        const float dr = (ru + rx > 0.f) ? (g.d0 / dim) / (ru + rx) : 0.f;
        return -20.f * expf(-0.2f * rx) * expm1f(-0.2f * dr) -
               2.71828182845904523536f * expf(-2.f * g.x1 / dim) * expm1f(-2.f * g.d1 / dim);
    }
    return g.d0;
}

// A whole row z[0..dim) held in shared memory, in blocks of S (lane s reads
// z[r0 + s], which must exist up to the row's padded length): f, with one
// dispatch on the objective per row instead of one per element.
template <int S, int OBJ>
__device__ __forceinline__ float group_obj_row_t(const float* z, int s, int dim) {
    GroupObj acc;
    for (int r0 = 0; r0 < dim; r0 += S) group_obj_push<S, OBJ>(OBJ, acc, z[r0 + s], r0, s, dim);
    return group_obj_finish<S>(OBJ, acc, dim);
}
template <int S>
__device__ __forceinline__ float group_obj_row(int obj, const float* z, int s, int dim) {
    switch (obj) {
    case kSphere: return group_obj_row_t<S, kSphere>(z, s, dim);
    case kRosenbrock: return group_obj_row_t<S, kRosenbrock>(z, s, dim);
    case kRastrigin: return group_obj_row_t<S, kRastrigin>(z, s, dim);
    case kGriewank: return group_obj_row_t<S, kGriewank>(z, s, dim);
    case kAckley: return group_obj_row_t<S, kAckley>(z, s, dim);
    default: return group_obj_row_t<S, kSchwefel12>(z, s, dim);
    }
}

// f(u) - f(x) from whole rows z and dz in shared memory, like group_obj_row.
template <int S, int OBJ>
__device__ __forceinline__ float group_diff_row_t(const float* z, const float* dz, int s, int dim) {
    GroupDiff g;
    for (int r0 = 0; r0 < dim; r0 += S) group_diff_push<S, OBJ>(OBJ, g, z[r0 + s], dz[r0 + s], r0, s, dim);
    return group_diff_finish<S>(OBJ, g, dim);
}
template <int S>
__device__ __forceinline__ float group_diff_row(int obj, const float* z, const float* dz, int s, int dim) {
    switch (obj) {
    case kSphere: return group_diff_row_t<S, kSphere>(z, dz, s, dim);
    case kRosenbrock: return group_diff_row_t<S, kRosenbrock>(z, dz, s, dim);
    case kRastrigin: return group_diff_row_t<S, kRastrigin>(z, dz, s, dim);
    case kGriewank: return group_diff_row_t<S, kGriewank>(z, dz, s, dim);
    case kAckley: return group_diff_row_t<S, kAckley>(z, dz, s, dim);
    default: return group_diff_row_t<S, kSchwefel12>(z, dz, s, dim);
    }
}

}  // namespace metade
