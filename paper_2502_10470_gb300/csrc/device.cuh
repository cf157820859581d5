// device.cuh -- device building blocks of the MetaDE generation step.
//
// Philox4x32-10 counter RNG (Salmon et al., SC'11), the per-individual draws
// of PDE (Sec. III-A: base vectors rand/best/pbest/current, dn difference
// vectors of distinct random individuals), crossover masks (Sec. II-A:
// binomial, exponential, arithmetic), and the synthetic shifted-rotated
// objectives in FP32 (numerically stable forms) and FP64.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace metade {

constexpr uint32_t kTagInner = 0x4D455441u;
constexpr uint32_t kTagOuter = 0x4F555445u;
constexpr uint32_t kInitGen = 0xFFFFFFFFu;
constexpr int kRecFields = 18;

// One executor, 64 bytes.  Offsets are in floats (population, padded
// problem tables) or elements (fitness).
struct InstDesc {
    long long pop_off;   // row 0 of the executor in the population
    long long rot_off;   // padded R [dim][dpad] (and R^T at the same offset in rotT)
    int fit_off;         // individual 0 in fitness arrays
    int np, dim, dpad;
    int obj, stream;     // objective id, Philox counter word 0
    int shift_off, kp;   // padded o [dpad]; pbest pool size
    int prob;            // problem index
    int tc_row;          // tensor-core / MLP path: first row of the executor in that path's row list
    int on_tc;           // 1: the executor is evaluated on the tensor-core path
    int aux;             // MLP objective: offset of the problem's targets [256][2]
};
static_assert(sizeof(InstDesc) == 64, "descriptor is one 64-byte record");

struct Key {
    uint32_t k0, k1;
};

__host__ __device__ inline Key make_key(uint64_t seed, uint32_t tag) {
    return Key{(uint32_t)seed, (uint32_t)(seed >> 32) ^ tag};
}

// Philox4x32, 10 rounds: the two multiplies feed a half swap, the key is
// mixed in and bumped by the Weyl increments (SC'11, Sec. 3.2).
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, Key k) {
    uint32_t k0 = k.k0, k1 = k.k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Counter = (stream, generation, individual, (epoch << 16) | slot).
struct Ctr {
    Key key;
    uint32_t stream, gen, indiv, epoch_hi;
    __device__ __forceinline__ uint4 slot(uint32_t s) const {
        return philox(stream, gen, indiv, epoch_hi | s, key);
    }
};

__device__ __forceinline__ Ctr make_ctr(Key key, uint32_t stream, uint32_t gen, uint32_t indiv, uint32_t epoch) {
    Ctr c;
    c.key = key;
    c.stream = stream;
    c.gen = gen;
    c.indiv = indiv;
    c.epoch_hi = epoch << 16;
    return c;
}

__device__ __forceinline__ uint32_t word_of(uint4 w, int q) {
    return q == 0 ? w.x : (q == 1 ? w.y : (q == 2 ? w.z : w.w));
}

// floor(w * m / 2^32): an integer in [0, m)
__device__ __forceinline__ uint32_t below(uint32_t w, uint32_t m) { return __umulhi(w, m); }

// 24-bit uniform (w >> 8) 2^-24, exact in float
__device__ __forceinline__ float uniform24(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

// U < p  <=>  (w >> 8) < ceil(p 2^24); p * 2^24 and its ceiling are exact in float.
__device__ __forceinline__ uint32_t threshold24(float p) {
    if (!(p > 0.0f)) return 0u;
    if (p >= 1.0f) return 16777216u;
    return (uint32_t)ceilf(p * 16777216.0f);
}

// ------------------------------------------------------------- strategy
struct Strat {
    float F, CR;
    int bl, br, dn, cs;
    uint32_t cri;
    int a, m;  // a = 1 when a rand base vector is used; m = a + 2 dn rand draws
    bool ok;
    __device__ __forceinline__ bool uses_pbest() const { return bl == 3 || br == 3; }
};

__device__ __forceinline__ Strat load_strat(const float* th, int np) {
    Strat s;
    s.F = th[0];
    s.CR = th[1];
    s.bl = (int)th[2];
    s.br = (int)th[3];
    s.dn = (int)th[4];
    s.cs = (int)th[5];
    s.a = (s.bl == 1 || s.br == 1) ? 1 : 0;
    s.m = s.a + 2 * s.dn;
    s.ok = isfinite(s.F) && isfinite(s.CR) && s.bl >= 1 && s.bl <= 4 && s.br >= 1 && s.br <= 4 &&
           s.dn >= 1 && s.dn <= 4 && s.cs >= 1 && s.cs <= 3 && np >= s.m + 1;
    if (!s.ok) {  // keep the arithmetic below well defined; the caller skips the executor
        s.bl = s.br = 4;
        s.dn = 1;
        s.cs = 1;
        s.a = 0;
        s.m = 2;
    }
    s.cri = threshold24(s.CR);
    return s;
}

// ------------------------------------------------------ individual draws
struct Indiv {
    int ibl, ibr;      // resolved base-left / base-right individuals
    int jrand, nstart; // binomial forced coordinate, exponential start
    int pbest;         // pbest individual (or -1 when the pool is not known)
    uint32_t kraw;     // K_i as a 24-bit integer
    int r[9];          // distinct rand draws r_0..r_{m-1}
};

// t-th draw: s = floor(w_t (np - 1 - t) / 2^32), then step s past the sorted
// excluded set {i, r_0..r_{t-1}}: the s-th smallest admissible index.
__device__ __forceinline__ void distinct_draws(int np, int i, int m, const uint32_t (&w)[12], int (&r)[9]) {
    int ex[10];
    ex[0] = i;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        r[t] = -1;
        if (t < m) {
            int v = (int)below(w[t], (uint32_t)(np - 1 - t));
#pragma unroll
            for (int e = 0; e < 10; ++e)
                if (e <= t && v >= ex[e]) ++v;
            r[t] = v;
            // insert v into ex[0..t] keeping it ascending
            bool placed = false;
#pragma unroll
            for (int e = 9; e >= 1; --e) {
                if (e <= t + 1 && !placed) {
                    if (ex[e - 1] > v) {
                        ex[e] = ex[e - 1];
                    } else {
                        ex[e] = v;
                        placed = true;
                    }
                }
            }
            if (!placed) ex[0] = v;
        }
    }
}

// Slot 0 words and the rand draws of individual i.  `topk` (the pbest pool,
// ascending by stored fitness) may be null when the strategy does not use it.
__device__ __forceinline__ void indiv_setup(const Strat& s, const Ctr& c, int i, int np, int dim, int kp,
                                            const int* topk, int best, Indiv& d) {
    const uint4 w0 = c.slot(0);
    const uint4 a = c.slot(1);  // m >= 2 always; independent of slot 0, so the two chains interleave
    d.jrand = (int)below(w0.x, (uint32_t)dim);
    d.nstart = (int)below(w0.y, (uint32_t)dim);
    d.kraw = w0.z >> 8;
    d.pbest = topk ? topk[below(w0.w, (uint32_t)kp)] : -1;
    uint32_t w[12];
    uint4 b = make_uint4(0, 0, 0, 0), e = b;
    if (s.m > 4) b = c.slot(2);
    if (s.m > 8) e = c.slot(3);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    w[8] = e.x; w[9] = e.y; w[10] = e.z; w[11] = e.w;
    distinct_draws(np, i, s.m, w, d.r);
    const int rb = d.r[0];
    d.ibl = s.bl == 1 ? rb : (s.bl == 2 ? best : (s.bl == 3 ? d.pbest : i));
    d.ibr = s.br == 1 ? rb : (s.br == 2 ? best : (s.br == 3 ? d.pbest : i));
}

// r index of difference q: plus-term (r[a + 2q]) and minus-term (r[a + 2q + 1])
__device__ __forceinline__ int diff_plus(const Indiv& d, int a, int q) {
    return a ? (q == 0 ? d.r[1] : q == 1 ? d.r[3] : q == 2 ? d.r[5] : d.r[7])
             : (q == 0 ? d.r[0] : q == 1 ? d.r[2] : q == 2 ? d.r[4] : d.r[6]);
}
__device__ __forceinline__ int diff_minus(const Indiv& d, int a, int q) {
    return a ? (q == 0 ? d.r[2] : q == 1 ? d.r[4] : q == 2 ? d.r[6] : d.r[8])
             : (q == 0 ? d.r[1] : q == 1 ? d.r[3] : q == 2 ? d.r[5] : d.r[7]);
}

// Exponential crossover length: L = 1, grow while L < D and the (L-1)-th
// coordinate uniform (slot 4 + (L-1)/4) is below CR.
__device__ __forceinline__ int exp_length(const Ctr& c, int dim, uint32_t cri) {
    int L = 1;
    for (uint32_t slot = 4; L < dim; ++slot) {
        const uint4 w = c.slot(slot);
        bool stop = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!stop && L < dim) {
                if ((word_of(w, q) >> 8) < cri) ++L;
                else stop = true;
            }
        }
        if (stop) break;
    }
    return L;
}

// exp_length by a whole warp (every lane returns L): lane l tests the uniforms
// t = base + 4 l .. base + 4 l + 3 (slot 4 + t / 4), 128 per round, and a
// ballot finds the first t <= D - 2 whose uniform is not below CR; then
// L = 1 + t, or D when there is none.  The same L as exp_length, in
// ceil((L - 1) / 128) rounds of one Philox call per lane instead of a chain
// of up to D / 4 calls.  Call with all 32 lanes, the same c, dim and cri.
__device__ __forceinline__ int warp_exp_length(const Ctr& c, int dim, uint32_t cri) {
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < dim - 1; base += 128) {
        const uint4 w = c.slot(4 + (uint32_t)(base >> 2) + (uint32_t)lane);
        int first = 4;  // this lane's first failing word
#pragma unroll
        for (int q = 3; q >= 0; --q) {
            const int t = base + 4 * lane + q;
            if (t <= dim - 2 && (word_of(w, q) >> 8) >= cri) first = q;
        }
        const unsigned fails = __ballot_sync(0xFFFFFFFFu, first < 4);
        if (fails) {
            const int fl = __ffs(fails) - 1;
            return 1 + base + 4 * fl + __shfl_sync(0xFFFFFFFFu, first, fl);
        }
    }
    return dim;
}

// ----------------------------------------------------------- objectives
// FP32 forms are algebraically equal to the textbook definitions but avoid
// cancellation near the optimum:
//   Rastrigin  z^2 - 10 cos 2 pi z + 10      = z^2 + 20 sin^2(pi z)
//   Ackley     20 + e - 20 e^{-0.2 r} - e^{C/D} = -20 expm1(-0.2 r) - e expm1(-2 S/D),
//              r = sqrt(sum z^2 / D), S = sum sin^2(pi z)
//   Griewank   1 - prod cos a_j = -expm1(sum log1p(-2 sin^2(a_j/2))) when every
//              cos a_j > 0, else evaluated directly (no cancellation then)
//   Rosenbrock y = z + 1: y_{j+1} - y_j^2 = z_{j+1} - z_j (z_j + 2), y_j - 1 = z_j
enum Obj { kSphere = 0, kRosenbrock = 1, kRastrigin = 2, kGriewank = 3, kAckley = 4, kSchwefel12 = 5, kMlp = 6 };

// MLP regression objective (6): the parameters of a 16-h-2 perceptron with
// one tanh hidden layer, W1 [16][h] (k h + j), b1 [h], W2 [h][2] (2 j + o),
// b2 [2], so D = 19 h + 2, against a teacher network (the problem's shift).
// f = mean over 256 fixed inputs and both outputs of the squared output
// difference.  Input n, coordinate k: 2 U - 1, U from Philox key
// (0, TAG_DATA), counter (0, 0, n, k / 4), word k % 4.
constexpr int kMlpIn = 16, kMlpOut = 2, kMlpN = 256;
constexpr uint32_t kTagData = 0x4D4C5044u;
__host__ __device__ inline int mlp_hidden(int dim) { return (dim >= 21 && (dim - 2) % 19 == 0) ? (dim - 2) / 19 : 0; }

// Network output for one input x: hidden units in order j = 0..h-1, each
// pre-activation summed over k ascending (fma), output accumulated over j.
// Four hidden units at a time when h % 4 == 0 (one float4 load of W1 feeds
// four fma chains; th must then be 16-byte aligned); the arithmetic of every
// unit and the order of the output sums are the same either way.
// T = float (FP32 evaluation) or double (FP64 evaluation).
template <typename T>
__device__ __forceinline__ void mlp_forward(int h, const float* th, const T (&x)[kMlpIn], T (&y)[kMlpOut]) {
    const float* W1 = th;
    const float* b1 = th + kMlpIn * h;
    const float* W2 = b1 + h;
    const float* b2 = W2 + kMlpOut * h;
    y[0] = T(b2[0]);
    y[1] = T(b2[1]);
    int j = 0;
    if ((h & 3) == 0) {
        for (; j < h; j += 4) {
            const float4 bb = *reinterpret_cast<const float4*>(b1 + j);
            T a[4] = {T(bb.x), T(bb.y), T(bb.z), T(bb.w)};
#pragma unroll
            for (int k = 0; k < kMlpIn; ++k) {
                const float4 w = *reinterpret_cast<const float4*>(W1 + k * h + j);
                a[0] = fma(x[k], T(w.x), a[0]);
                a[1] = fma(x[k], T(w.y), a[1]);
                a[2] = fma(x[k], T(w.z), a[2]);
                a[3] = fma(x[k], T(w.w), a[3]);
            }
            const float4 w2a = *reinterpret_cast<const float4*>(W2 + 2 * j);
            const float4 w2b = *reinterpret_cast<const float4*>(W2 + 2 * j + 4);
            const float v2[8] = {w2a.x, w2a.y, w2a.z, w2a.w, w2b.x, w2b.y, w2b.z, w2b.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const T t = tanh(a[q]);
                y[0] = fma(t, T(v2[2 * q]), y[0]);
                y[1] = fma(t, T(v2[2 * q + 1]), y[1]);
            }
        }
    }
    for (; j < h; ++j) {
        T a = T(b1[j]);
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) a = fma(x[k], T(W1[k * h + j]), a);
        const T t = tanh(a);
        y[0] = fma(t, T(W2[2 * j]), y[0]);
        y[1] = fma(t, T(W2[2 * j + 1]), y[1]);
    }
}

// The same forward pass for two inputs at once: every weight load feeds both
// (each input's arithmetic is exactly that of mlp_forward).  FP32 only.
__device__ __forceinline__ void mlp_forward2(int h, const float* th, const float (&xa)[kMlpIn],
                                             const float (&xb)[kMlpIn], float (&ya)[kMlpOut],
                                             float (&yb)[kMlpOut]) {
    if ((h & 3) != 0) {
        mlp_forward<float>(h, th, xa, ya);
        mlp_forward<float>(h, th, xb, yb);
        return;
    }
    const float* W1 = th;
    const float* b1 = th + kMlpIn * h;
    const float* W2 = b1 + h;
    const float* b2 = W2 + kMlpOut * h;
    ya[0] = yb[0] = b2[0];
    ya[1] = yb[1] = b2[1];
    for (int j = 0; j < h; j += 4) {
        const float4 bb = *reinterpret_cast<const float4*>(b1 + j);
        float a[4] = {bb.x, bb.y, bb.z, bb.w}, c[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) {
            const float4 w = *reinterpret_cast<const float4*>(W1 + k * h + j);
            a[0] = fmaf(xa[k], w.x, a[0]);
            a[1] = fmaf(xa[k], w.y, a[1]);
            a[2] = fmaf(xa[k], w.z, a[2]);
            a[3] = fmaf(xa[k], w.w, a[3]);
            c[0] = fmaf(xb[k], w.x, c[0]);
            c[1] = fmaf(xb[k], w.y, c[1]);
            c[2] = fmaf(xb[k], w.z, c[2]);
            c[3] = fmaf(xb[k], w.w, c[3]);
        }
        const float4 w2a = *reinterpret_cast<const float4*>(W2 + 2 * j);
        const float4 w2b = *reinterpret_cast<const float4*>(W2 + 2 * j + 4);
        const float v2[8] = {w2a.x, w2a.y, w2a.z, w2a.w, w2b.x, w2b.y, w2b.z, w2b.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float ta = tanhf(a[q]), tb = tanhf(c[q]);
            ya[0] = fmaf(ta, v2[2 * q], ya[0]);
            ya[1] = fmaf(ta, v2[2 * q + 1], ya[1]);
            yb[0] = fmaf(tb, v2[2 * q], yb[0]);
            yb[1] = fmaf(tb, v2[2 * q + 1], yb[1]);
        }
    }
}

// Streaming accumulator: objectives consume z_0, z_1, ... in order.
template <typename T>
struct ObjAcc {
    T s0, s1, s2, prev;
    int n;
    bool pos;
};

template <typename T>
__device__ __forceinline__ T sinpi_t(T x);
template <>
__device__ __forceinline__ float sinpi_t<float>(float x) { return sinpif(x); }
template <>
__device__ __forceinline__ double sinpi_t<double>(double x) { return sinpi(x); }

template <typename T>
__device__ __forceinline__ void obj_init(ObjAcc<T>& a) {
    a.s0 = T(0); a.s1 = T(0); a.s2 = T(0); a.prev = T(0); a.n = 0; a.pos = true;
}

template <typename T>
__device__ __forceinline__ void obj_push(int obj, ObjAcc<T>& a, T z) {
    switch (obj) {
    case kSphere: a.s0 += z * z; break;
    case kRosenbrock:
        if (a.n > 0) {
            const T t = z - a.prev * (a.prev + T(2));
            a.s0 += T(100) * t * t + a.prev * a.prev;
        }
        a.prev = z;
        break;
    case kRastrigin: {
        const T s = sinpi_t<T>(z);
        a.s0 += z * z + T(20) * s * s;
        break;
    }
    case kGriewank: {
        a.s0 += z * z;
        const T arg = z / sqrt(T(a.n + 1));
        const T h = sin(arg * T(0.5));
        a.s1 += log1p(T(-2) * h * h);
        const T c = cos(arg);
        a.pos = a.pos && (c > T(0));
        a.s2 = (a.n == 0) ? c : a.s2 * c;
        break;
    }
    case kAckley: {
        a.s0 += z * z;
        const T s = sinpi_t<T>(z);
        a.s1 += s * s;
        break;
    }
    case kSchwefel12:
        a.prev += z;
        a.s0 += a.prev * a.prev;
        break;
    }
    ++a.n;
}

template <typename T>
__device__ __forceinline__ T obj_finish(int obj, const ObjAcc<T>& a, int dim) {
    switch (obj) {
    case kGriewank: {
        const T one_minus_p = a.pos ? -expm1(a.s1) : (T(1) - a.s2);
        return a.s0 / T(4000) + one_minus_p;
    }
    case kAckley: {
        const T r = sqrt(a.s0 / T(dim));
        return T(-20) * expm1(T(-0.2) * r) - T(2.71828182845904523536) * expm1(T(-2) * a.s1 / T(dim));
    }
    default: return a.s0;
    }
}

// 1/pi and 1/(2 pi) as floats: angles are passed in units of pi to sin_pi,
// sincos_pi and sin2pi, whose range reduction (x - rint(x)) is exact.
constexpr float kInvPi = 0.318309886f;
constexpr float kInv2Pi = 0.159154943f;

// sin^2(pi x) in FP32: t = x - rint(x) (exact), u = t^2, and
// sin^2(pi t) = u P(u) with P of degree 5 fitted to sin^2(pi sqrt(u)) / u on
// [0, 1/4] in the relative sense (weighted least squares driven toward the
// minimax error; fit error 1.4e-8).  Relative error of the FP32 evaluation
// below 2.2e-7 over all x: that of a correctly rounded sin(pi x), squared.
__device__ __forceinline__ float sin2pi(float x) {
    const float t = x - rintf(x);
    const float u = t * t;
    float p = -3.336236715e+00f;
    p = fmaf(p, u, 1.303712845e+01f);
    p = fmaf(p, u, -3.009855652e+01f);
    p = fmaf(p, u, 4.272692871e+01f);
    p = fmaf(p, u, -3.246966171e+01f);
    p = fmaf(p, u, 9.869604111e+00f);
    return u * p;
}

// sin(pi x) and cos(pi x) in FP32: n = rint(x), t = x - n (exact), u = t^2,
// sin(pi t) = t S(u) and cos(pi t) = C(u) with S, C of degree 5 fitted on
// [0, 1/4] to sin(pi sqrt u) / sqrt u (relative) and cos(pi sqrt u)
// (absolute), then the sign of (-1)^n (n odd iff n / 2 is not an integer,
// exact at every magnitude).  Errors below 2.1e-7 relative (sin) and 1.4e-7
// absolute (cos).
__device__ __forceinline__ bool odd_int(float n) { return 0.5f * n != rintf(0.5f * n); }
__device__ __forceinline__ float sin_pi(float x) {
    const float n = rintf(x), t = x - n, u = t * t;
    float p = -7.022167556e-03f;
    p = fmaf(p, u, 8.204647899e-02f);
    p = fmaf(p, u, -5.992513299e-01f);
    p = fmaf(p, u, 2.550163269e+00f);
    p = fmaf(p, u, -5.167712688e+00f);
    p = fmaf(p, u, 3.141592741e+00f);
    const float v = t * p;
    return odd_int(n) ? -v : v;
}
__device__ __forceinline__ void sincos_pi(float x, float* sp, float* cp) {
    const float n = rintf(x), t = x - n, u = t * t;
    float ps = -7.022167556e-03f;
    ps = fmaf(ps, u, 8.204647899e-02f);
    ps = fmaf(ps, u, -5.992513299e-01f);
    ps = fmaf(ps, u, 2.550163269e+00f);
    ps = fmaf(ps, u, -5.167712688e+00f);
    ps = fmaf(ps, u, 3.141592741e+00f);
    float pc = -2.439673804e-02f;
    pc = fmaf(pc, u, 2.349375784e-01f);
    pc = fmaf(pc, u, -1.335212111e+00f);
    pc = fmaf(pc, u, 4.058709145e+00f);
    pc = fmaf(pc, u, -4.934802055e+00f);
    pc = fmaf(pc, u, 1.0f);
    const bool odd = odd_int(n);
    const float sv = t * ps;
    *sp = odd ? -sv : sv;
    *cp = odd ? -pc : pc;
}

// FP32 objective streaming over z_0, z_1, ... with the objective chosen at run
// time (one code path for all objectives keeps the fused kernel's instruction
// footprint small).  Griewank uses the telescoping form
// 1 - prod c_j = sum_j (1 - c_j) prod_{k<j} c_k with
// 1 - c_j = 2 sin^2(a_j / 2), a_j = z_j / sqrt(j), and sin(a_j / 2) taken as
// sinpi(z_j k_j), k_j = 1 / (2 pi sqrt(j)) (the caller's per-coordinate
// argument): one transcendental per coordinate and no cancellation near the
// optimum.
struct ObjR {
    float s0 = 0.f, s1 = 0.f, prev = 0.f, pre = 1.f;
    bool first = true;
    // One coordinate, objective fixed at compile time (no per-element switch,
    // so independent elements of an unrolled block interleave).
    template <int OBJ>
    __device__ __forceinline__ void push_t(float z, float kj) {
        if constexpr (OBJ == kSphere) {
            s0 = fmaf(z, z, s0);
        } else if constexpr (OBJ == kRosenbrock) {
            if (!first) {
                const float t = z - prev * (prev + 2.f);
                s0 += 100.f * t * t + prev * prev;
            }
            prev = z;
            first = false;
        } else if constexpr (OBJ == kRastrigin) {
            s0 += z * z + 20.f * sin2pi(z);
        } else if constexpr (OBJ == kGriewank) {
            s0 = fmaf(z, z, s0);
            const float w = 2.f * sin2pi(z * kj);
            s1 = fmaf(pre, w, s1);
            pre *= 1.f - w;
        } else if constexpr (OBJ == kAckley) {
            s0 = fmaf(z, z, s0);
            s1 += sin2pi(z);
        } else {
            prev += z;
            s0 = fmaf(prev, prev, s0);
        }
    }
    __device__ __forceinline__ void push(int obj, float z, float kj) {
        switch (obj) {
        case kSphere: push_t<kSphere>(z, kj); break;
        case kRosenbrock: push_t<kRosenbrock>(z, kj); break;
        case kRastrigin: push_t<kRastrigin>(z, kj); break;
        case kGriewank: push_t<kGriewank>(z, kj); break;
        case kAckley: push_t<kAckley>(z, kj); break;
        default: push_t<kSchwefel12>(z, kj); break;
        }
    }
    // Four consecutive coordinates, one dispatch.
    template <int OBJ>
    __device__ __forceinline__ void push4_t(float z0, float z1, float z2, float z3, const float* isq) {
        push_t<OBJ>(z0, isq[0]);
        push_t<OBJ>(z1, isq[1]);
        push_t<OBJ>(z2, isq[2]);
        push_t<OBJ>(z3, isq[3]);
    }
    __device__ __forceinline__ void push4(int obj, float z0, float z1, float z2, float z3, const float* isq) {
        switch (obj) {
        case kSphere: push4_t<kSphere>(z0, z1, z2, z3, isq); break;
        case kRosenbrock: push4_t<kRosenbrock>(z0, z1, z2, z3, isq); break;
        case kRastrigin: push4_t<kRastrigin>(z0, z1, z2, z3, isq); break;
        case kGriewank: push4_t<kGriewank>(z0, z1, z2, z3, isq); break;
        case kAckley: push4_t<kAckley>(z0, z1, z2, z3, isq); break;
        default: push4_t<kSchwefel12>(z0, z1, z2, z3, isq); break;
        }
    }
    // 32 consecutive coordinates col0.. (those below dim), in order; a block
    // wholly below dim (every block of a row but its last) without the test
    // per coordinate.
    template <int OBJ>
    __device__ __forceinline__ void push32_t(const float (&v)[32], int col0, int dim) {
        if (col0 + 32 <= dim) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                push_t<OBJ>(v[j], OBJ == kGriewank ? rsqrtf((float)(col0 + j + 1)) * kInv2Pi : 0.f);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (col0 + j < dim)
                    push_t<OBJ>(v[j], OBJ == kGriewank ? rsqrtf((float)(col0 + j + 1)) * kInv2Pi : 0.f);
        }
    }
    // push32_t for Griewank with the factors of coordinates col0 .. col0 + 31
    // read from kj[0 ..] (a table holding rsqrtf(j + 1) * kInv2Pi, the values
    // push32_t computes, so the state is the same)
    __device__ __forceinline__ void push32_griewank(const float (&v)[32], int col0, int dim, const float* kj) {
        if (col0 + 32 <= dim) {
#pragma unroll
            for (int j = 0; j < 32; ++j) push_t<kGriewank>(v[j], kj[j]);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (col0 + j < dim) push_t<kGriewank>(v[j], kj[j]);
        }
    }
    __device__ __forceinline__ void push32(int obj, const float (&v)[32], int col0, int dim) {
        switch (obj) {
        case kSphere: push32_t<kSphere>(v, col0, dim); break;
        case kRosenbrock: push32_t<kRosenbrock>(v, col0, dim); break;
        case kRastrigin: push32_t<kRastrigin>(v, col0, dim); break;
        case kGriewank: push32_t<kGriewank>(v, col0, dim); break;
        case kAckley: push32_t<kAckley>(v, col0, dim); break;
        default: push32_t<kSchwefel12>(v, col0, dim); break;
        }
    }
    __device__ __forceinline__ float finish(int obj, int dim) const {
        if (obj == kGriewank) return s0 * (1.f / 4000.f) + s1;
        if (obj == kAckley)
            return -20.f * expm1f(-0.2f * sqrtf(s0 / dim)) - 2.71828182845904523536f * expm1f(-2.f * s1 / dim);
        return s0;
    }
};

__device__ __forceinline__ float nan_to_inf(float f) { return isnan(f) ? INFINITY : f; }
__device__ __forceinline__ double nan_to_inf(double f) { return isnan(f) ? (double)INFINITY : f; }

// Sequential FP64 evaluation of one float32 point (selection ties, FP64
// evaluation).  o: padded shift, R: padded rows [dim][dpad].
__device__ __forceinline__ double eval64_seq(int obj, int dim, int dpad, const float* x, const float* o,
                                             const float* R) {
    ObjAcc<double> a;
    obj_init(a);
    for (int r = 0; r < dim; ++r) {
        double z = 0.0;
        const float* row = R + (size_t)r * dpad;
        for (int c = 0; c < dim; ++c) z = fma((double)row[c], (double)x[c] - (double)o[c], z);
        obj_push(obj, a, z);
    }
    return obj_finish(obj, a, dim);
}

// cos(a + 2h) - cos(a) = -2 sin(a + h) sin(h), with sin(a + h) expanded as
// sin a cos h + cos a sin h so that one sincos_pi(a / pi) serves both terms;
// sin h and cos h come from their Taylor series when |h| <= 1/16 (relative
// error below 1e-9) and from sincos_pi otherwise.  Writes cos(a) to c.
__device__ __forceinline__ float cos_step(float a, float h, float& c) {
    float sa, ca, sh, ch;
    sincos_pi(a * kInvPi, &sa, &ca);
    if (fabsf(h) <= 0.0625f) {
        const float h2 = h * h;
        sh = h * (1.f - h2 * (1.f / 6.f) * (1.f - h2 * (1.f / 20.f)));
        ch = 1.f - 0.5f * h2 * (1.f - h2 * (1.f / 12.f));
    } else {
        sincos_pi(h * kInvPi, &sh, &ch);
    }
    c = ca;
    return -2.f * (sa * ch + ca * sh) * sh;
}

// ----------------------------------------------------- tie differences
// Selection ties are decided on D = f(u) - f(x) evaluated directly as a
// difference, from z = R (x - o) and dz = R (u - x), so that its rounding
// error scales with |D| instead of |f|:
//   z^2 terms        (z+dz)^2 - z^2            = dz (2 z + dz)
//   sin^2 terms      sin^2(pi(z+dz)) - sin^2(pi z) = sin(pi(2z+dz)) sin(pi dz)
//   Rosenbrock t     t' - t = dz_{j+1} - dz_j (2 z_j + 2 + dz_j)
//   Schwefel prefix  p' - p = running sum of dz
//   Griewank product P' - P by D_n = c'_n D_{n-1} + (c'_n - c_n) P_{n-1},
//                    c' - c = -2 sin(a + da/2) sin(da/2)
//   Ackley           r' - r = (r'^2 - r^2) / (r' + r);  e^{-c r} - e^{-c r'} =
//                    -e^{-c r} expm1(-c (r' - r)), likewise for the cosine mean.
struct DiffAcc {
    float d0, d1, x0, x1;  // difference sums, x-side sums
    float pz, pdz;         // previous z, dz (Rosenbrock)
    float p, dp;           // prefix of z, dz (Schwefel 1.2)
    float lr, px;          // Griewank: product difference D_n, product P_n
    int n;
};

__device__ __forceinline__ void diff_init(DiffAcc& a) {
    a.d0 = a.d1 = a.x0 = a.x1 = 0.f;
    a.pz = a.pdz = a.p = a.dp = 0.f;
    a.lr = 0.f;
    a.px = 1.f;
    a.n = 0;
}

__device__ __forceinline__ void diff_push(int obj, DiffAcc& a, float z, float dz) {
    switch (obj) {
    case kSphere: a.d0 += dz * (2.f * z + dz); break;
    case kRosenbrock:
        if (a.n > 0) {
            const float t = z - a.pz * (a.pz + 2.f);
            const float dt = dz - a.pdz * (2.f * a.pz + 2.f + a.pdz);
            a.d0 += 100.f * dt * (2.f * t + dt) + a.pdz * (2.f * a.pz + a.pdz);
        }
        a.pz = z;
        a.pdz = dz;
        break;
    case kRastrigin:
        a.d0 += dz * (2.f * z + dz) + 20.f * sin_pi(2.f * z + dz) * sin_pi(dz);
        break;
    case kGriewank: {
        // product difference by the telescoping recurrence
        //   D_n = c'_n D_{n-1} + (c'_n - c_n) P_{n-1},  P_n = P_{n-1} c_n,
        //   c' - c = cos(a + da) - cos(a) = -2 sin(a + da/2) sin(da/2)
        a.d0 += dz * (2.f * z + dz);
        const float inv = rsqrtf((float)(a.n + 1));
        const float ang = z * inv, da = dz * inv;
        const float dc = cos_step(ang, 0.5f * da, a.pz);  // pz receives cos(ang)
        a.lr = (a.pz + dc) * a.lr + dc * a.px;            // lr holds D_n, px holds P_n
        a.px *= a.pz;
        break;
    }
    case kAckley: {
        a.x0 += z * z;
        a.d0 += dz * (2.f * z + dz);
        a.x1 += sin2pi(z);
        a.d1 += sin_pi(2.f * z + dz) * sin_pi(dz);
        break;
    }
    case kSchwefel12:
        a.p += z;
        a.dp += dz;
        a.d0 += a.dp * (2.f * a.p + a.dp);
        break;
    }
    ++a.n;
}

__device__ __forceinline__ float diff_finish(int obj, const DiffAcc& a, int dim) {
    switch (obj) {
    case kGriewank: return a.d0 / 4000.f - a.lr;
    case kAckley: {
        const float rx = sqrtf(a.x0 / dim), ru = sqrtf(fmaxf(a.x0 + a.d0, 0.f) / dim);
        const float dr = (ru + rx > 0.f) ? (a.d0 / dim) / (ru + rx) : 0.f;
        return -20.f * expf(-0.2f * rx) * expm1f(-0.2f * dr) -
               2.71828182845904523536f * expf(-2.f * a.x1 / dim) * expm1f(-2.f * a.d1 / dim);
    }
    default: return a.d0;
    }
}

// Sequential difference f(u) - f(x) of two float32 points (rows of length
// dim, shift o, padded rows R with stride ldr).
__device__ __forceinline__ float diff_seq(int obj, int dim, int ldr, const float* u, const float* x, const float* o,
                                          const float* R) {
    DiffAcc a;
    diff_init(a);
    for (int r = 0; r < dim; ++r) {
        const float* row = R + (size_t)r * ldr;
        float z = 0.f, dz = 0.f;
        for (int c = 0; c < dim; ++c) {
            z = fmaf(row[c], x[c] - o[c], z);
            dz = fmaf(row[c], u[c] - x[c], dz);
        }
        diff_push(obj, a, z, dz);
    }
    return diff_finish(obj, a, dim);
}

// Selection ties: |f(u) - f(x)| <= band |f(x)| with both values finite and
// positive are decided by the FP32 difference form or an FP64 re-evaluation,
// not by the two FP32 values.  band(D) = max(1e-6, 2^-21 sqrt(D)): the 1e-6
// band of the requirement, widened where the FP32 error of f itself grows
// like sqrt(D) ulps (at D = 200 Schwefel 1.2 reaches 1.8e-6 relative, about
// 2 sqrt(D) ulps; 2^-21 sqrt(D) = 8 sqrt(D) ulps leaves a factor of four).
// The band is relative: FP32 resolves f to a fixed relative precision at any
// magnitude, and an absolute floor would send every trial of a converged
// executor down the tie path.  Values that underflowed to 0 compare as equal
// and the trial wins.
__host__ __device__ __forceinline__ float tie_band(int dim) {
    return fmaxf(1e-6f, 4.76837158203125e-7f * sqrtf((float)dim));
}
__device__ __forceinline__ bool near_tie(float fu, float fx, float band) {
    return isfinite(fu) && isfinite(fx) && fx > 0.0f && fu > 0.0f && fabsf(fu - fx) <= band * fx;
}

// Sticky device status: the first error wins.
__device__ __forceinline__ void set_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

}  // namespace metade
