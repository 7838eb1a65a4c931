// Shared device helpers: complex arithmetic on float2/double2, deterministic
// block reductions, float <-> double conversions and two-float arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nk {

template <typename R> struct C2;
template <> struct C2<float> { typedef float2 T; };
template <> struct C2<double> { typedef double2 T; };

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
    return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return mk(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return mk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__host__ __device__ __forceinline__ double cnorm2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double2 cinv(double2 a) {
    // 1/a with Smith's scaling to avoid overflow in |a|^2
    if (fabs(a.x) >= fabs(a.y)) {
        double r = a.y / a.x, d = a.x + a.y * r;
        return mk(1.0 / d, -r / d);
    } else {
        double r = a.x / a.y, d = a.x * r + a.y;
        return mk(r / d, -1.0 / d);
    }
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) { return cmul(a, cinv(b)); }
// principal square root (cut on the negative real axis)
__host__ __device__ __forceinline__ double2 csqrt_principal(double2 z) {
    double r = hypot(z.x, z.y);
    if (r == 0.0) return mk(0.0, 0.0);
    double t = sqrt(0.5 * (r + fabs(z.x)));
    if (z.x >= 0.0) return mk(t, z.y / (2.0 * t));
    return mk(fabs(z.y) / (2.0 * t), z.y >= 0.0 ? t : -t);
}

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
__device__ __forceinline__ double2 to_d2(float2 a) { return mk((double)a.x, (double)a.y); }

// Warp sum of a double2 in a fixed butterfly order (deterministic).
__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Linear thread index and thread count of the block (blocks may be 2-D with
// blockDim.x a multiple of 32: warps are then runs of 32 linear indices).
__device__ __forceinline__ int block_tid() { return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z); }
__device__ __forceinline__ int block_threads() { return blockDim.x * blockDim.y * blockDim.z; }

// Block sum of a double2 (<= 1024 threads in whole warps). Every thread of the
// block receives the same value; the summation order is fixed.  Only warp 0
// does the second level (FP64 adds are scarce on GB300); the result is
// broadcast through shared memory.  The butterfly of the second level stops at
// the number of warps (lanes beyond it hold zeros).
__device__ __forceinline__ double2 block_sum(double2 v, double2* sh /* >= 33 */) {
    v = warp_sum(v);
    const int tid = block_tid();
    int lane = tid & 31, w = tid >> 5, nw = block_threads() >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        double2 t = lane < nw ? sh[lane] : mk(0.0, 0.0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            if (o < nw) {   // only the levels that combine real partials
                t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
                t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
            }
        }
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}
__device__ __forceinline__ double block_sum(double v, double* sh /* >= 32 */) {
    v = warp_sum(v);
    const int tid = block_tid();
    int lane = tid & 31, w = tid >> 5, nw = block_threads() >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
    return t;
}

// Two-stage deterministic reduction, stage 1: thread 0 of each block writes
// its block's partial; the block that arrives last (integer ticket, no
// floating-point atomics) returns true and finishes the sum in fixed order.
__device__ __forceinline__ bool finish_partial(double2 part, double2* partials, unsigned* counter,
                                               int slot, int nslots) {
    __shared__ bool last;
    if (block_tid() == 0) {
        partials[slot] = part;
        __threadfence();
        unsigned ticket = atomicAdd(counter, 1u);
        last = (ticket == (unsigned)nslots - 1u);
    }
    __syncthreads();
    return last;
}

// Stage 2: fixed-order sum of the nslots partials (all threads of the last block).
__device__ __forceinline__ double2 sum_partials(const double2* partials, int nslots, double2* sh) {
    __threadfence();
    double2 a = mk(0.0, 0.0);
    for (int i = block_tid(); i < nslots; i += block_threads()) {
        double2 v = __ldcg(partials + i);
        a.x += v.x; a.y += v.y;
    }
    return block_sum(a, sh);
}

// ---- float <-> double on the integer pipe ---------------------------------------
// On GB300 the FP64 pipe is 1/64 of the FP32 rate and cvt.f64.f32 /
// cvt.f32.f64 issue on it too, so the hot kernels move between the formats
// with integer bit operations only (IEEE 754 binary32 <-> binary64 field
// layout), with no conversion instruction even on a predicated-off path.
// Normal numbers and zero convert exactly / round to nearest; the edge cases
// the vectors of this method never reach are mapped without a conversion
// instruction: float subnormals and double results below the normal float
// range become signed zero, overflow becomes infinity, NaN stays NaN.

// float -> double, exact for normal floats and zero
__device__ __forceinline__ double f2d_int(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned s = u & 0x80000000u;
    const unsigned a = u & 0x7fffffffu;
    unsigned hi = s | ((a >> 3) + (896u << 20));
    unsigned lo = a << 29;
    if (a < 0x00800000u) { hi = s; lo = 0u; }                        // zero, subnormal -> 0
    if (a >= 0x7f800000u) { hi = s | 0x7ff00000u | ((a >> 3) & 0x000fffffu); }   // inf / NaN
    return __hiloint2double((int)hi, (int)lo);
}

// double -> float, rounded to nearest (ties away from zero in magnitude; ties
// occur with probability 2^-29 and differ from round-to-even by one ulp).
// Every range check is made on the 32-bit high word: checks on the 64-bit
// pattern of |d| were turned by the compiler into FP64 comparisons, which
// issue on the scarce FP64 pipe.
__device__ __forceinline__ float d2f_int(double d) {
    const unsigned h = (unsigned)__double2hiint(d), l = (unsigned)__double2loint(d);
    const unsigned s = h & 0x80000000u, ah = h & 0x7fffffffu;
    // (wraps around below the normal float range; the underflow rule is applied last)
    const unsigned t = (((ah - (896u << 20)) << 3) | (l >> 29)) + ((l >> 28) & 1u);
    unsigned r = t;
    if (ah >= (1151u << 20) || t >= (255u << 23)) r = 0x7f800000u;             // overflow -> inf
    if (ah < (897u << 20)) r = 0u;                                               // below normal floats -> 0
    if (ah > 0x7ff00000u || (ah == 0x7ff00000u && l != 0u)) r = 0x7fc00000u;     // NaN
    return __uint_as_float(s | r);
}

// double -> (hi, lo) floats with hi + lo == d to about 2^-48 relative: hi is d
// truncated to 24 significant bits (exact in float), lo the remaining 29 bits
// rounded to a float.  Outside the normal float range: (d2f_int(d), 0).
__device__ __forceinline__ float2 d2ff_int(double d) {
    const unsigned h = (unsigned)__double2hiint(d), l = (unsigned)__double2loint(d);
    const unsigned s = h & 0x80000000u, ah = h & 0x7fffffffu;
    const unsigned e = ah >> 20;
    const bool normal = ah >= (897u << 20) && ah < (1151u << 20);
    float hi = __uint_as_float(s | (((ah - (896u << 20)) << 3) | (l >> 29)));
    const unsigned mlo = l & 0x1fffffffu;                                        // d - hi = mlo * 2^(e - 1075)
    float lo = __uint2float_rn(mlo) * __uint_as_float(((e > 948u ? e : 949u) - 948u) << 23);
    lo = __uint_as_float(__float_as_uint(lo) | s);
    if (e <= 948u) lo = 0.0f;
    if (!normal) { hi = d2f_int(d); lo = 0.0f; }
    return make_float2(hi, lo);
}

// ---- two-float ("df") arithmetic ---------------------------------------------------
// A value is hi + lo with |lo| <= ulp(hi); about 48 significant bits, computed
// on the FP32 pipe with the error-free transformations TwoSum (Knuth) and
// TwoProd via FMA (the double-float arithmetic of Dekker and of Hida, Li and
// Bailey's double-double library).  The _rn intrinsics keep the compiler from
// contracting or reassociating the steps.
struct df {
    float hi, lo;
    __host__ __device__ __forceinline__ df() {}
    __host__ __device__ __forceinline__ df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ __forceinline__ df(int v) : hi((float)v), lo(0.0f) {}
};
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df operator+(df a, df b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(s, e);
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { a = a + b; return a; }
__device__ __forceinline__ df df_from_double(double d) {
    const float2 p = d2ff_int(d);
    return df(p.x, p.y);
}
__device__ __forceinline__ double df_to_double(df a) { return f2d_int(a.hi) + f2d_int(a.lo); }

struct __align__(16) dfc {
    df x, y;
};

// Unnormalised two-float accumulator: the value is s + e, with |e| small
// against |s| but not renormalised after each step.  Adding an exact product
// (TwoProd via FMA, including the cross terms of two-float operands) or
// another value is TwoSum on the leading parts and a plain FP32 sum of the
// trailing parts: 12 and 8 FP32 instructions, against 18 and 11 for the
// normalised product and sum (the accumulation of Ogita, Rump and Oishi's
// compensated dot product, applied to two-float operands).  dfa_value
// renormalises once at the end.
struct dfa {
    float s, e;
};
__device__ __forceinline__ dfa dfa_of(df a) { return {a.hi, a.lo}; }
__device__ __forceinline__ dfa dfa_neg(dfa a) { return {-a.s, -a.e}; }
// (ah + al) (bh + bl) up to the al bl term
__device__ __forceinline__ dfa dfa_prod(float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    return {p, e};
}
// a += s + e
__device__ __forceinline__ void dfa_add(dfa& a, float s, float e) {
    const float t = __fadd_rn(a.s, s);
    const float v = __fsub_rn(t, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, v)), __fsub_rn(s, v));
    a.s = t;
    a.e = __fadd_rn(a.e, __fadd_rn(e, err));
}
__device__ __forceinline__ void dfa_add(dfa& a, dfa b) { dfa_add(a, b.s, b.e); }
__device__ __forceinline__ void dfa_add_prod(dfa& a, float ah, float al, float bh, float bl) {
    const dfa p = dfa_prod(ah, al, bh, bl);
    dfa_add(a, p.s, p.e);
}
__device__ __forceinline__ df dfa_value(dfa a) { return df_fast_two_sum(a.s, a.e); }
struct dfac {
    dfa x, y;
};
template <> struct C2<df> { typedef dfc T; };
static_assert(sizeof(dfc) == 16, "two-float complex is 16 bytes");

}  // namespace nk
