// Packed two-lane FP32 arithmetic of sm_100+ (add/sub/mul/fma .rn.f32x2 in
// inline PTX): one instruction applies the same FP32 operation, each lane
// rounded to nearest, to two floats held in one 64-bit register.  The
// two-float stencil keeps its values in this form.
#pragma once

namespace nk {

typedef unsigned long long f2p;   // two floats: lane 0 in the low word

__device__ __forceinline__ f2p pk(float a, float b) {
    f2p r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2p v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2p swp(f2p v) {   // (a, b) -> (b, a)
    float a, b;
    upk(v, a, b);
    return pk(b, a);
}
// lane-wise sign flips: -x in both lanes, and in lane 0 or lane 1 only (exact)
__device__ __forceinline__ f2p neg2(f2p v) { return v ^ 0x8000000080000000ull; }
__device__ __forceinline__ f2p neg_lo(f2p v) { return v ^ 0x0000000080000000ull; }
__device__ __forceinline__ f2p neg_hi(f2p v) { return v ^ 0x8000000000000000ull; }

__device__ __forceinline__ f2p add2(f2p a, f2p b) {
    f2p d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p sub2(f2p a, f2p b) {
    f2p d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p mul2(f2p a, f2p b) {
    f2p d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// ---- two-float values, two lanes at a time -----------------------------------
// A value is s + e per lane; |e| is small against |s| but the pair is not
// renormalised after each step (the unnormalised accumulation of the scalar
// two-float code, nk_common.cuh, lane-wise: TwoSum of Knuth and TwoProd via
// FMA, with the trailing parts summed in plain FP32).
struct P2 {
    f2p s, e;
};

// a + b (the leading parts by TwoSum, the trailing ones plainly added)
__device__ __forceinline__ P2 p2_add(P2 a, P2 b) {
    const f2p t = add2(a.s, b.s);
    const f2p v = sub2(t, a.s);
    const f2p err = add2(sub2(a.s, sub2(t, v)), sub2(b.s, v));
    return {t, add2(add2(a.e, b.e), err)};
}
// (a.s + a.e)(b.s + b.e) up to the a.e b.e term: TwoProd of the leading
// parts plus the cross terms in FP32
__device__ __forceinline__ P2 p2_prod(P2 a, P2 b) {
    const f2p p = mul2(a.s, b.s);
    f2p e = fma2(a.s, b.s, neg2(p));
    e = fma2(a.s, b.e, e);
    e = fma2(a.e, b.s, e);
    return {p, e};
}
// acc += a b
__device__ __forceinline__ void p2_add_prod(P2& acc, P2 a, P2 b) { acc = p2_add(acc, p2_prod(a, b)); }
__device__ __forceinline__ P2 p2_neg(P2 a) { return {neg2(a.s), neg2(a.e)}; }
__device__ __forceinline__ P2 p2_swp(P2 a) { return {swp(a.s), swp(a.e)}; }
// lane signs: (-a0, a1) and (a0, -a1)
__device__ __forceinline__ P2 p2_neg_lo(P2 a) { return {neg_lo(a.s), neg_lo(a.e)}; }
__device__ __forceinline__ P2 p2_neg_hi(P2 a) { return {neg_hi(a.s), neg_hi(a.e)}; }

}  // namespace nk
