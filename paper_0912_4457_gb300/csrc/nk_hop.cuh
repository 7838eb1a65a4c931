// The Wilson hop of Sec. 2 in the chiral basis, for FP32 and FP64 values in
// registers: acc += w (1 + s gamma_nu) M psi with M = U or U^dagger.  Shared
// by the stencil kernels of dslash.cu and stencil32.cu.
//
// (1 + s gamma_nu) psi = [h ; s B_nu h] with the half spinor
// h = psi_up + s C_nu psi_dn, C_k = -i sigma_k, B_k = i sigma_k, C_4 = B_4 = 1,
// so each hop multiplies only the two colour vectors of h by the link.
#pragma once

#include "nk_common.cuh"

namespace nk {

// a * b + c with one rounding (FFMA / DFMA): the stencil's sums are written as
// chains of these, since `x += a * b - c * d` compiles to a multiply, a fused
// multiply-add and an add -- three instructions for two products
__device__ __forceinline__ float mac(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mac(double a, double b, double c) { return fma(a, b, c); }

// i * z and -i * z
template <typename T> __device__ __forceinline__ T mul_i(T z) { T r; r.x = -z.y; r.y = z.x; return r; }
template <typename T> __device__ __forceinline__ T mul_mi(T z) { T r; r.x = z.y; r.y = -z.x; return r; }
template <typename T> __device__ __forceinline__ T neg(T z) { T r; r.x = -z.x; r.y = -z.y; return r; }

// One hop: acc += w * (1 + s gamma_nu) M psi_n with M = U (dag = false) or
// U^dagger, from a neighbour spinor and link already loaded into registers
// (FP32 and FP64; the two-float stencil has its own form below).
template <int NU, bool DAG, typename R>
__device__ __forceinline__ void hop_regs(typename C2<R>::T acc[4][3], const typename C2<R>::T psi[4][3],
                                         const typename C2<R>::T u[3][3], R s, R w) {
    typedef typename C2<R>::T T;
    T h0[3], h1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T c0, c1;  // (C_nu psi_dn)_0, _1
        if (NU == 0) { c0 = mul_mi(psi[3][a]); c1 = mul_mi(psi[2][a]); }
        else if (NU == 1) { c0 = neg(psi[3][a]); c1 = psi[2][a]; }
        else if (NU == 2) { c0 = mul_mi(psi[2][a]); c1 = mul_i(psi[3][a]); }
        else { c0 = psi[2][a]; c1 = psi[3][a]; }
        h0[a].x = mac(s, c0.x, psi[0][a].x); h0[a].y = mac(s, c0.y, psi[0][a].y);
        h1[a].x = mac(s, c1.x, psi[1][a].x); h1[a].y = mac(s, c1.y, psi[1][a].y);
    }
    const R ws = w * s;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T x0, x1;
        x0.x = 0; x0.y = 0; x1.x = 0; x1.y = 0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const T e = DAG ? u[b][a] : u[a][b];
            const R ey = DAG ? -e.y : e.y;
            x0.x = mac(e.x, h0[b].x, x0.x); x0.x = mac(-ey, h0[b].y, x0.x);
            x0.y = mac(e.x, h0[b].y, x0.y); x0.y = mac(ey, h0[b].x, x0.y);
            x1.x = mac(e.x, h1[b].x, x1.x); x1.x = mac(-ey, h1[b].y, x1.x);
            x1.y = mac(e.x, h1[b].y, x1.y); x1.y = mac(ey, h1[b].x, x1.y);
        }
        acc[0][a].x = mac(w, x0.x, acc[0][a].x); acc[0][a].y = mac(w, x0.y, acc[0][a].y);
        acc[1][a].x = mac(w, x1.x, acc[1][a].x); acc[1][a].y = mac(w, x1.y, acc[1][a].y);
        T b0, b1;  // (B_nu m)_0, _1
        if (NU == 0) { b0 = mul_i(x1); b1 = mul_i(x0); }
        else if (NU == 1) { b0 = x1; b1 = neg(x0); }
        else if (NU == 2) { b0 = mul_i(x0); b1 = mul_mi(x1); }
        else { b0 = x0; b1 = x1; }
        acc[2][a].x = mac(ws, b0.x, acc[2][a].x); acc[2][a].y = mac(ws, b0.y, acc[2][a].y);
        acc[3][a].x = mac(ws, b1.x, acc[3][a].x); acc[3][a].y = mac(ws, b1.y, acc[3][a].y);
    }
}

}  // namespace nk
