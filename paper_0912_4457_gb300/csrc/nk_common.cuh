// Shared device helpers: complex arithmetic on float2/double2, deterministic
// block reductions, the bounded-wait policy.
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

// Block sum of a double2 (blockDim.x a multiple of 32, <= 1024). Every thread
// of the block receives the same value; the summation order is fixed.
__device__ __forceinline__ double2 block_sum(double2 v, double2* sh /* >= 32 */) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double2 t = lane < nw ? sh[lane] : mk(0.0, 0.0);
    t = warp_sum(t);
    return t;
}
__device__ __forceinline__ double block_sum(double v, double* sh /* >= 32 */) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
    return t;
}

// Upper bound on spin iterations of any device-side wait (each iteration
// sleeps ~100 ns), about one second; a wait that runs out sets an error flag.
constexpr long long kSpinLimit = 10000000LL;

}  // namespace nk
