// Wilson-Dirac stencil A = gamma5 D_w(mu) and A^dagger = gamma5 D_w(-mu).
//
// D_w(mu) of Sec. 2: (D_w psi)_y = psi_y
//     - kappa sum_nu w+_nu (1 + gamma_nu) U_{y-nu,+nu} psi_{y-nu}
//     - kappa sum_nu w-_nu (1 - gamma_nu) U^dagger_{y,+nu} psi_{y+nu},
// w+-_nu = 1 for nu = x,y,z and w+_t = e^{mu}, w-_t = e^{-mu}; a hop across
// the t boundary carries a factor -1 (antiperiodic).  Since
// gamma5 D_w(mu) gamma5 = D_w(-mu)^dagger, A^dagger = gamma5 D_w(-mu): the same
// stencil with the two temporal weights exchanged, so one kernel serves the
// right (A v) and left (A^dagger w) recurrences of the two-sided Lanczos
// process in a single launch, reading each link once for both.
//
// Chiral basis: (1 + s gamma_nu) psi = [h ; s B_nu h] with the half spinor
// h = psi_up + s C_nu psi_dn, C_k = -i sigma_k, B_k = i sigma_k, C_4 = B_4 = 1,
// so each hop multiplies only the two colour vectors of h by the link.
//
// Layouts (device-internal, set up by the engine):
//   links:   [nu 4][e 9][site V] complex, e = 3*row + col (coalesced over sites)
//   spinors: [component 12][site V] complex per vector, component = 3*spin + colour
#include <type_traits>

#include "nk_common.cuh"
#include "nk_hop.cuh"
#include "nk_kernels.h"

namespace nk {

template <typename R>
struct Spinor {
    typename C2<R>::T c[4][3];
};

template <typename R>
__device__ __forceinline__ void load_spinor(const typename C2<R>::T* __restrict__ in, int V, int site,
                                            typename C2<R>::T p[4][3]) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) p[s][a] = in[(size_t)(3 * s + a) * V + site];
}

template <typename R>
__device__ __forceinline__ void load_link(const typename C2<R>::T* __restrict__ U, int V, int nu, int site,
                                          typename C2<R>::T u[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) u[a][b] = U[(size_t)(nu * 9 + 3 * a + b) * V + site];
}

template <int NU, typename R>
__device__ __forceinline__ void dir(typename C2<R>::T acc[4][3], const typename C2<R>::T* __restrict__ U,
                                    const typename C2<R>::T* __restrict__ in, const Geom& g, int site,
                                    int coord, int L, int stride, R wplus, R wminus) {
    // backward neighbour y - nu: (1 + gamma) U_{y-nu,+nu} psi_{y-nu}
    typedef typename C2<R>::T T;
    const int sb = coord == 0 ? site + (L - 1) * stride : site - stride;
    const R fb = (NU == 3 && g.antiperiodic && coord == 0) ? R(-1) : R(1);
    const int sf = coord == L - 1 ? site - (L - 1) * stride : site + stride;
    const R ff = (NU == 3 && g.antiperiodic && coord == L - 1) ? R(-1) : R(1);
    T u[3][3], p[4][3];
    load_link<R>(U, g.V, NU, sb, u);
    load_spinor<R>(in, g.V, sb, p);
    hop_regs<NU, false, R>(acc, p, u, R(1), wplus * fb);
    // forward neighbour y + nu: (1 - gamma) U^dagger_{y,+nu} psi_{y+nu}
    load_link<R>(U, g.V, NU, site, u);
    load_spinor<R>(in, g.V, sf, p);
    hop_regs<NU, true, R>(acc, p, u, R(-1), wminus * ff);
}

// ---- colour split: one thread per (site, colour a) -----------------------------
// The same hop restricted to row a of M psi: the thread projects the whole
// neighbour spinor (all three colours) but forms and accumulates only the a-th
// row, so it holds a quarter of the accumulators; three threads share a site.
template <int NU, bool DAG, typename R>
__device__ __forceinline__ void hop_regs_a(typename C2<R>::T acc[4], const typename C2<R>::T psi[4][3],
                                           const typename C2<R>::T urow[3], R s, R w) {
    typedef typename C2<R>::T T;
    T h0[3], h1[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        T c0, c1;
        if (NU == 0) { c0 = mul_mi(psi[3][b]); c1 = mul_mi(psi[2][b]); }
        else if (NU == 1) { c0 = neg(psi[3][b]); c1 = psi[2][b]; }
        else if (NU == 2) { c0 = mul_mi(psi[2][b]); c1 = mul_i(psi[3][b]); }
        else { c0 = psi[2][b]; c1 = psi[3][b]; }
        h0[b].x = psi[0][b].x + s * c0.x; h0[b].y = psi[0][b].y + s * c0.y;
        h1[b].x = psi[1][b].x + s * c1.x; h1[b].y = psi[1][b].y + s * c1.y;
    }
    const R ws = w * s;
    T x0, x1;
    x0.x = 0; x0.y = 0; x1.x = 0; x1.y = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const T e = urow[b];
        R ey = DAG ? -e.y : e.y;
        x0.x += e.x * h0[b].x - ey * h0[b].y; x0.y += e.x * h0[b].y + ey * h0[b].x;
        x1.x += e.x * h1[b].x - ey * h1[b].y; x1.y += e.x * h1[b].y + ey * h1[b].x;
    }
    acc[0].x += w * x0.x; acc[0].y += w * x0.y;
    acc[1].x += w * x1.x; acc[1].y += w * x1.y;
    T b0, b1;
    if (NU == 0) { b0 = mul_i(x1); b1 = mul_i(x0); }
    else if (NU == 1) { b0 = x1; b1 = neg(x0); }
    else if (NU == 2) { b0 = mul_i(x0); b1 = mul_mi(x1); }
    else { b0 = x0; b1 = x1; }
    acc[2].x += ws * b0.x; acc[2].y += ws * b0.y;
    acc[3].x += ws * b1.x; acc[3].y += ws * b1.y;
}

template <int NU, typename R>
__device__ __forceinline__ void dir_a(typename C2<R>::T acc[4], const typename C2<R>::T* __restrict__ U,
                                      const typename C2<R>::T* __restrict__ in, const Geom& g, int site, int a,
                                      int coord, int L, int stride, R wplus, R wminus) {
    typedef typename C2<R>::T T;
    const int sb = coord == 0 ? site + (L - 1) * stride : site - stride;
    const R fb = (NU == 3 && g.antiperiodic && coord == 0) ? R(-1) : R(1);
    const int sf = coord == L - 1 ? site - (L - 1) * stride : site + stride;
    const R ff = (NU == 3 && g.antiperiodic && coord == L - 1) ? R(-1) : R(1);
    T urow[3], p[4][3];
#pragma unroll
    for (int b = 0; b < 3; ++b) urow[b] = U[(size_t)(NU * 9 + 3 * a + b) * g.V + sb];   // row a of U
    load_spinor<R>(in, g.V, sb, p);
    hop_regs_a<NU, false, R>(acc, p, urow, R(1), wplus * fb);
#pragma unroll
    for (int b = 0; b < 3; ++b) urow[b] = U[(size_t)(NU * 9 + 3 * b + a) * g.V + site]; // column a: row a of U^dagger
    load_spinor<R>(in, g.V, sf, p);
    hop_regs_a<NU, true, R>(acc, p, urow, R(-1), wminus * ff);
}

// ---- the two-float stencil: one copy of the hop body --------------------------
// Two-float arithmetic turns every flop into 7-11 FP32 instructions; the
// eight hops unrolled with compile-time gamma structure then overflow the
// instruction cache (ncu: most stalls "no instruction").  Here the eight hops
// run as a loop over one hop body: the direction is a warp-uniform run-time
// value and the gamma matrices act through multiplications by i^q (exact:
// swaps and sign changes), so the values are those of the unrolled form.
__device__ __forceinline__ dfc rot_q(dfc z, int q) {   // z * i^q
    dfc r;
    switch (q & 3) {
        case 0: r = z; break;
        case 1: r.x = -z.y; r.y = z.x; break;
        case 2: r.x = -z.x; r.y = -z.y; break;
        default: r.x = z.y; r.y = -z.x; break;
    }
    return r;
}
// (C_nu psi)_0 = i^q0 psi_{i0}, (C_nu psi)_1 = i^q1 psi_{i1}; (B_nu m)_0 = i^r0q m_{r0},
// (B_nu m)_1 = i^r1q m_{r1} -- the chiral-basis structure of the unrolled hop
struct HopSpin { int i0, q0, i1, q1, r0, r0q, r1, r1q; };
__device__ __forceinline__ HopSpin hop_spin(int nu) {
    switch (nu) {
        case 0: return {3, 3, 2, 3, 1, 1, 0, 1};
        case 1: return {3, 2, 2, 0, 1, 0, 0, 2};
        case 2: return {2, 3, 3, 1, 0, 1, 1, 3};
        default: return {2, 0, 3, 0, 0, 0, 1, 0};
    }
}

__device__ __forceinline__ dfac rot_q(dfac z, int q) {   // z * i^q
    dfac r;
    switch (q & 3) {
        case 0: r = z; break;
        case 1: r.x = dfa_neg(z.y); r.y = z.x; break;
        case 2: r.x = dfa_neg(z.x); r.y = dfa_neg(z.y); break;
        default: r.x = z.y; r.y = dfa_neg(z.x); break;
    }
    return r;
}

// Neighbour index, link site and two-float weight of hop h (nu = h / 2; odd h:
// forward neighbour, (1 - gamma) U^dagger_{y,+nu} psi_{y+nu}).
struct HopGeo { int sn, ls; df w; };
__device__ __forceinline__ HopGeo hop_geo(const Geom& g, int site, const int coord[4], int h, df wp_t,
                                          df wm_t) {
    const int nu = h >> 1;
    const bool fwd = (h & 1) != 0;
    int L, stride;
    switch (nu) {
        case 0: L = g.Lx; stride = 1; break;
        case 1: L = g.Ly; stride = g.Lx; break;
        case 2: L = g.Lz; stride = g.Lx * g.Ly; break;
        default: L = g.Lt; stride = g.Lx * g.Ly * g.Lz; break;
    }
    const int c = coord[nu];
    HopGeo r;
    bool wrap;
    if (fwd) { wrap = c == L - 1; r.sn = wrap ? site - (L - 1) * stride : site + stride; r.ls = site; }
    else { wrap = c == 0; r.sn = wrap ? site + (L - 1) * stride : site - stride; r.ls = r.sn; }
    const df flip = (nu == 3 && g.antiperiodic && wrap) ? df(-1) : df(1);
    r.w = (nu == 3 ? (fwd ? wm_t : wp_t) : df(1)) * flip;
    return r;
}

// Half spinors h0, h1 of one hop (the projection: additions of +-1 and +-i
// multiples, exact up to the two-float rounding).
__device__ __forceinline__ void hop_project(dfac h0[3], dfac h1[3], const dfc* __restrict__ in, int V, int sn,
                                            const HopSpin& hs, bool fwd) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const dfc p0 = in[(size_t)b * V + sn], p1 = in[(size_t)(3 + b) * V + sn];
        const dfc p2 = in[(size_t)(6 + b) * V + sn], p3 = in[(size_t)(9 + b) * V + sn];
        const dfc c0 = rot_q(hs.i0 == 3 ? p3 : p2, fwd ? hs.q0 + 2 : hs.q0);   // -c for the forward hop
        const dfc c1 = rot_q(hs.i1 == 3 ? p3 : p2, fwd ? hs.q1 + 2 : hs.q1);
        h0[b].x = dfa_of(p0.x); dfa_add(h0[b].x, c0.x.hi, c0.x.lo);
        h0[b].y = dfa_of(p0.y); dfa_add(h0[b].y, c0.y.hi, c0.y.lo);
        h1[b].x = dfa_of(p1.x); dfa_add(h1[b].x, c1.x.hi, c1.x.lo);
        h1[b].y = dfa_of(p1.y); dfa_add(h1[b].y, c1.y.hi, c1.y.lo);
    }
}

// Row a of the link (or of its adjoint, forward hops) times h0 and h1: each
// output component is a dot product of six two-float products, accumulated
// unnormalised; nu = t multiplies by the temporal weight.  Adds the results
// to the four spin components of acc (colour a).
__device__ __forceinline__ void hop_row(dfac acc[4], const dfc* __restrict__ U, int V, int ls, int nu, bool fwd,
                                        int a, const dfac h0[3], const dfac h1[3], const HopSpin& hs, df w) {
    dfac x0, x1;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const int e_idx = fwd ? nu * 9 + 3 * b + a : nu * 9 + 3 * a + b;
        const dfc e = U[(size_t)e_idx * V + ls];
        const float eyh = fwd ? -e.y.hi : e.y.hi, eyl = fwd ? -e.y.lo : e.y.lo;
        if (b == 0) {
            x0.x = dfa_prod(e.x.hi, e.x.lo, h0[0].x.s, h0[0].x.e);
            x0.y = dfa_prod(e.x.hi, e.x.lo, h0[0].y.s, h0[0].y.e);
            x1.x = dfa_prod(e.x.hi, e.x.lo, h1[0].x.s, h1[0].x.e);
            x1.y = dfa_prod(e.x.hi, e.x.lo, h1[0].y.s, h1[0].y.e);
        } else {
            dfa_add_prod(x0.x, e.x.hi, e.x.lo, h0[b].x.s, h0[b].x.e);
            dfa_add_prod(x0.y, e.x.hi, e.x.lo, h0[b].y.s, h0[b].y.e);
            dfa_add_prod(x1.x, e.x.hi, e.x.lo, h1[b].x.s, h1[b].x.e);
            dfa_add_prod(x1.y, e.x.hi, e.x.lo, h1[b].y.s, h1[b].y.e);
        }
        dfa_add_prod(x0.x, -eyh, -eyl, h0[b].y.s, h0[b].y.e);
        dfa_add_prod(x0.y, eyh, eyl, h0[b].x.s, h0[b].x.e);
        dfa_add_prod(x1.x, -eyh, -eyl, h1[b].y.s, h1[b].y.e);
        dfa_add_prod(x1.y, eyh, eyl, h1[b].x.s, h1[b].x.e);
    }
    if (nu == 3) {   // temporal weights e^{+-mu} and the boundary sign
        x0.x = dfa_prod(x0.x.s, x0.x.e, w.hi, w.lo);
        x0.y = dfa_prod(x0.y.s, x0.y.e, w.hi, w.lo);
        x1.x = dfa_prod(x1.x.s, x1.x.e, w.hi, w.lo);
        x1.y = dfa_prod(x1.y.s, x1.y.e, w.hi, w.lo);
    }
    dfa_add(acc[0].x, x0.x); dfa_add(acc[0].y, x0.y);
    dfa_add(acc[1].x, x1.x); dfa_add(acc[1].y, x1.y);
    const dfac b0 = rot_q(hs.r0 == 1 ? x1 : x0, fwd ? hs.r0q + 2 : hs.r0q);   // times -1 forward
    const dfac b1 = rot_q(hs.r1 == 1 ? x1 : x0, fwd ? hs.r1q + 2 : hs.r1q);
    dfa_add(acc[2].x, b0.x); dfa_add(acc[2].y, b0.y);
    dfa_add(acc[3].x, b1.x); dfa_add(acc[3].y, b1.y);
}

__device__ __forceinline__ dfc dfc_value(dfac a) {
    dfc r;
    r.x = dfa_value(a.x);
    r.y = dfa_value(a.y);
    return r;
}

// The sum over the eight hops of one site, all colours (acc[spin][colour]).
__device__ __forceinline__ void stencil_hops_df(dfc acc[4][3], const dfc* __restrict__ U, const dfc* __restrict__ in,
                                                const Geom& g, int site, const int coord[4], df wp_t, df wm_t) {
    const int V = g.V;
    dfac A[3][4];   // [colour][spin], unnormalised
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) A[a][sp].x = A[a][sp].y = dfa{0.0f, 0.0f};
#pragma unroll 1
    for (int h = 0; h < 8; ++h) {
        const int nu = h >> 1;
        const bool fwd = (h & 1) != 0;
        const HopGeo hg = hop_geo(g, site, coord, h, wp_t, wm_t);
        const HopSpin hs = hop_spin(nu);
        dfac h0[3], h1[3];
        hop_project(h0, h1, in, V, hg.sn, hs, fwd);
#pragma unroll
        for (int a = 0; a < 3; ++a) hop_row(A[a], U, V, hg.ls, nu, fwd, a, h0, h1, hs, hg.w);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) acc[sp][a] = dfc_value(A[a][sp]);
}

// The same for colour a only (three threads per site).
__device__ __forceinline__ void stencil_hops_df_a(dfc acc[4], const dfc* __restrict__ U, const dfc* __restrict__ in,
                                                  const Geom& g, int site, int a, const int coord[4], df wp_t,
                                                  df wm_t) {
    const int V = g.V;
    dfac A[4];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) A[sp].x = A[sp].y = dfa{0.0f, 0.0f};
#pragma unroll 1
    for (int h = 0; h < 8; ++h) {
        const int nu = h >> 1;
        const bool fwd = (h & 1) != 0;
        const HopGeo hg = hop_geo(g, site, coord, h, wp_t, wm_t);
        const HopSpin hs = hop_spin(nu);
        dfac h0[3], h1[3];
        hop_project(h0, h1, in, V, hg.sn, hs, fwd);
        hop_row(A, U, V, hg.ls, nu, fwd, a, h0, h1, hs, hg.w);
    }
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) acc[sp] = dfc_value(A[sp]);
}

// precision-generic conversions (float via the integer pipe, see nk_common.cuh)
__device__ __forceinline__ double to_double(float a) { return f2d_int(a); }
__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double to_double(df a) { return df_to_double(a); }
template <typename R> __device__ __forceinline__ R from_double(double d);
template <> __device__ __forceinline__ float from_double<float>(double d) { return d2f_int(d); }
template <> __device__ __forceinline__ double from_double<double>(double d) { return d; }
template <> __device__ __forceinline__ df from_double<df>(double d) { return df_from_double(d); }
// two-float complex values for the mixed-schedule epilogue
__device__ __forceinline__ dfc to_dfc(float2 v) {
    dfc r;
    r.x = df(v.x, 0.0f);
    r.y = df(v.y, 0.0f);
    return r;
}
__device__ __forceinline__ dfc to_dfc(dfc v) { return v; }
__device__ __forceinline__ dfc dfc_of2(double2 v) {
    dfc r;
    r.x = df_from_double(v.x);
    r.y = df_from_double(v.y);
    return r;
}
// a two-float kernel argument from a host double
static df df_host(double d) {
    df r;
    r.hi = (float)d;
    r.lo = (float)(d - (double)r.hi);
    return r;
}
// s - c p and s + c p with explicit FMA (4 FP64 instructions each)
__device__ __forceinline__ double2 caxpy_neg(double2 s, double2 c, double2 p) {
    return make_double2(fma(-c.x, p.x, fma(c.y, p.y, s.x)), fma(-c.x, p.y, fma(-c.y, p.x, s.y)));
}
__device__ __forceinline__ double2 caxpy_pos(double2 s, double2 c, double2 p) {
    return make_double2(fma(c.x, p.x, fma(-c.y, p.y, s.x)), fma(c.x, p.y, fma(c.y, p.x, s.y)));
}

// out = gamma5 (psi - kappa * hops)(site) for one vector: A psi (dag = 0) or
// A^dagger psi = gamma5 D_w(-mu) psi (dag = 1), in precision R.
template <typename R>
__device__ __forceinline__ void stencil_site(const typename C2<R>::T* __restrict__ U,
                                             const typename C2<R>::T* __restrict__ in, const Geom& g,
                                             int site, int dag, R kappa, R emu, R emu_inv,
                                             typename C2<R>::T out[4][3]) {
    typedef typename C2<R>::T T;
    // temporal weights: A uses (e^{mu}, e^{-mu}); A^dagger exchanges them
    const R wp_t = dag ? emu_inv : emu;
    const R wm_t = dag ? emu : emu_inv;
    int x = site % g.Lx;
    int r = site / g.Lx;
    int y = r % g.Ly; r /= g.Ly;
    int z = r % g.Lz;
    int t = r / g.Lz;
    T acc[4][3];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) { acc[sp][a].x = 0; acc[sp][a].y = 0; }
    if constexpr (std::is_same<R, df>::value) {
        const int coord[4] = {x, y, z, t};
        stencil_hops_df(acc, U, in, g, site, coord, wp_t, wm_t);
    } else {
        dir<0, R>(acc, U, in, g, site, x, g.Lx, 1, R(1), R(1));
        dir<1, R>(acc, U, in, g, site, y, g.Ly, g.Lx, R(1), R(1));
        dir<2, R>(acc, U, in, g, site, z, g.Lz, g.Lx * g.Ly, R(1), R(1));
        dir<3, R>(acc, U, in, g, site, t, g.Lt, g.Lx * g.Ly * g.Lz, wp_t, wm_t);
    }
    T p[4][3];
    load_spinor<R>(in, g.V, site, p);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
        const R sg = sp < 2 ? R(1) : R(-1);  // gamma5 = diag(1, 1, -1, -1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            out[sp][a].x = sg * (p[sp][a].x - kappa * acc[sp][a].x);
            out[sp][a].y = sg * (p[sp][a].y - kappa * acc[sp][a].y);
        }
    }
}

// The colour-a components of gamma5 (psi - kappa * hops)(site): out[sp] for colour a.
template <typename R>
__device__ __forceinline__ void stencil_site_a(const typename C2<R>::T* __restrict__ U,
                                               const typename C2<R>::T* __restrict__ in, const Geom& g,
                                               int site, int a, int dag, R kappa, R emu, R emu_inv,
                                               typename C2<R>::T out[4]) {
    typedef typename C2<R>::T T;
    const R wp_t = dag ? emu_inv : emu;
    const R wm_t = dag ? emu : emu_inv;
    int x = site % g.Lx;
    int r = site / g.Lx;
    int y = r % g.Ly; r /= g.Ly;
    int z = r % g.Lz;
    int t = r / g.Lz;
    T acc[4];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) { acc[sp].x = 0; acc[sp].y = 0; }
    if constexpr (std::is_same<R, df>::value) {
        const int coord[4] = {x, y, z, t};
        stencil_hops_df_a(acc, U, in, g, site, a, coord, wp_t, wm_t);
    } else {
        dir_a<0, R>(acc, U, in, g, site, a, x, g.Lx, 1, R(1), R(1));
        dir_a<1, R>(acc, U, in, g, site, a, y, g.Ly, g.Lx, R(1), R(1));
        dir_a<2, R>(acc, U, in, g, site, a, z, g.Lz, g.Lx * g.Ly, R(1), R(1));
        dir_a<3, R>(acc, U, in, g, site, a, t, g.Lt, g.Lx * g.Ly * g.Lz, wp_t, wm_t);
    }
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
        const R sg = sp < 2 ? R(1) : R(-1);
        const T p = in[(size_t)(3 * sp + a) * g.V + site];
        out[sp].x = sg * (p.x - kappa * acc[sp].x);
        out[sp].y = sg * (p.y - kappa * acc[sp].y);
    }
}

// One thread per (site, vector). Vectors [0, n0) come from set 0, [n0, n0+n1)
// from set 1; set s applies A (dag = 0) or A^dagger (dag = 1).
template <typename R>
__global__ void __launch_bounds__(128) dslash_kernel(const typename C2<R>::T* __restrict__ U, Geom g,
                                                      DslashSet s0, DslashSet s1, R kappa, R emu, R emu_inv) {
    typedef typename C2<R>::T T;
    const int nvec = s0.n + s1.n;
    const int vec = blockIdx.x % nvec;
    const int site = (blockIdx.x / nvec) * blockDim.x + threadIdx.x;
    if (site >= g.V) return;
    const DslashSet& S = vec < s0.n ? s0 : s1;
    const int vi = vec < s0.n ? vec : vec - s0.n;
    const T* __restrict__ in = reinterpret_cast<const T*>(S.in) + (size_t)vi * S.in_stride;
    double2* __restrict__ out = S.out + (size_t)vi * S.out_stride;
    T o[4][3];
    stencil_site<R>(U, in, g, site, S.dag, kappa, emu, emu_inv, o);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            out[(size_t)(3 * sp + a) * g.V + site] = make_double2(to_double(o[sp][a].x), to_double(o[sp][a].y));
}

void launch_dslash(int precision, const void* U, const Geom& g, const DslashSet& s0,
                   const DslashSet& s1, double kappa, double mu, cudaStream_t st) {
    const int threads = 128;
    const int nvec = s0.n + s1.n;
    if (nvec == 0) return;
    dim3 grid((unsigned)(((g.V + threads - 1) / threads) * nvec));
    if (precision == 48)
        dslash_kernel<df><<<grid, threads, 0, st>>>((const dfc*)U, g, s0, s1, df_host(kappa), df_host(exp(mu)),
                                                   df_host(exp(-mu)));
    else
        dslash_kernel<double><<<grid, threads, 0, st>>>((const double2*)U, g, s0, s1, kappa, exp(mu), exp(-mu));
}

// ---- fused stencil + first half of an outer Lanczos step ------------------------
//
// For outer step j (see lanczos.cu for the unnormalised basis q_j, p_j):
//   right vectors (side 0, one per RHS):
//     s = A q_j / n_j;  r = s - (c_{j-1}/n_{j-1}) q_{j-1}  (c = beta, two-sided gamma)
//     r -> q_{j+1};  partial of H(j,j) = v_j^dag r  (two-sided w_j^dag r)
//   left vectors (side 1, two-sided only):
//     t = A^dag p_j / m_j;  l = t - (beta^*_{j-1}/m_{j-1}) p_{j-1};  l -> p_{j+1}
// The stencil runs in precision R (FP32 reads the FP32 copies of q_j, p_j and
// the FP32 links; the two-float stencil reads the two-float rings); the scale
// 1/n_j of its output is part of the stencil application (A v_j = A q_j / n_j)
// and is applied in the same precision.  The rest of the epilogue (the
// update with q_{j-1}, p_{j-1} and the H(j,j) partial) runs in FP64 on the
// FP64 vectors, or, from step o.ring_from on (the optional two-float
// recurrence of the mixed schedule), in two-float arithmetic on the rings.  The blocks of side 0 reduce H(j,j) with the deterministic
// two-stage scheme.  In double-pass mode side 0 also accumulates
// y += c'_j q_j at its own site.
// Minimum resident CTAs of kStencilMaxThreads threads per SM for the fused
// stencil (a register cap): the FP32 and two-float instantiations are
// latency bound (loads; long dependent FP32 chains) and gain from more
// resident warps than their unconstrained register counts (about 160) allow.
template <typename R> struct StencilMinBlocks { static constexpr int value = 1; };
template <> struct StencilMinBlocks<df> { static constexpr int value = 2; };
template <> struct StencilMinBlocks<float> { static constexpr int value = 3; };

// CS: threads per site (1, or 3 with one colour each; blockDim = (sites, CS)).
template <typename R, bool TS, bool PASS2, int CS>
__global__ void __launch_bounds__(CS * kStencilMaxThreads, CS == 1 ? StencilMinBlocks<R>::value : 1) k_dslash_step1(
    const typename C2<R>::T* __restrict__ U, Geom g, Outer o, int j, R kappa, R emu, R emu_inv,
    const typename C2<R>::T* __restrict__ qin, long qin_stride, const typename C2<R>::T* __restrict__ pin,
    long pin_stride) {
    typedef typename C2<R>::T T;
    __shared__ double2 sh[33];
    __shared__ double2 coef[3];
    const int nvec = TS ? 2 * o.n_rhs : o.n_rhs;
    const int nsb = gridDim.x / nvec;
    const int vec = o.st_order == 0 ? blockIdx.x % nvec : blockIdx.x / nsb;
    const int sb = o.st_order == 0 ? blockIdx.x / nvec : blockIdx.x % nsb;
    const int side = vec / o.n_rhs;      // 0: A q_j, 1: A^dagger p_j
    const int rhs = vec % o.n_rhs;
    if (o.status[rhs] != kStatusOK) return;
    if (side == 1 && j == o.k - 1) return;   // the last step needs no left vector
    const size_t hb = (size_t)rhs * o.k;
    // the scalars of this step (a complex FP64 division or inverse each), one
    // per warp so that they run side by side instead of one after another
    if ((block_tid() & 31) == 0) {
        const int nw = block_threads() >> 5;   // 2 warps or more
        for (int t = block_tid() >> 5; t < 3; t += nw) {
            const double2 zero = make_double2(0.0, 0.0);
            double2 v;
            if (side == 0) {
                if (t == 0) v = cinv(scale_n(o, rhs, j));
                else if (t == 1) v = j > 0 ? cdiv(TS ? o.gamma[hb + j - 1] : o.beta[hb + j - 1], scale_n(o, rhs, j - 1)) : zero;
                else v = TS ? cinv(cconj(scale_m(o, rhs, j))) : cinv(scale_n(o, rhs, j));
            } else {
                if (t == 0) v = cinv(scale_m(o, rhs, j));
                else if (t == 1) v = j > 0 ? cdiv(cconj(o.beta[hb + j - 1]), scale_m(o, rhs, j - 1)) : zero;
                else v = zero;
            }
            coef[t] = v;
        }
    }
    __syncthreads();
    const int site = sb * blockDim.x + threadIdx.x;
    double2 acc = make_double2(0.0, 0.0);
    if (site < g.V) {
        const T* __restrict__ in = side == 0 ? qin + (size_t)rhs * qin_stride : pin + (size_t)rhs * pin_stride;
        // the stencil output of this thread's components, handed to epi(sp, a, value)
        auto for_each_out = [&](auto&& epi) {
            if constexpr (CS == 1) {
                T out[4][3];
                stencil_site<R>(U, in, g, site, side, kappa, emu, emu_inv, out);
#pragma unroll
                for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                    for (int a = 0; a < 3; ++a) epi(sp, a, out[sp][a]);
            } else {
                const int a = threadIdx.y;
                T out[4];
                stencil_site_a<R>(U, in, g, site, a, side, kappa, emu, emu_inv, out);
#pragma unroll
                for (int sp = 0; sp < 4; ++sp) epi(sp, a, out[sp]);
            }
        };
        const double2 c1 = coef[1];   // zero at j = 0 (the previous vector is then any valid one)
        const int jp = j > 0 ? j - 1 : j;
        bool ring_epilogue = false;
        if constexpr (!std::is_same<R, double>::value) ring_epilogue = j >= o.ring_from;
        if constexpr (!std::is_same<R, double>::value) if (ring_epilogue) {
            // steps of the mixed schedule from ring_from on (the two-float
            // recurrence): the epilogue in two-float arithmetic on the rings
            const dfc scr = dfc_of2(coef[0]), c1d = dfc_of2(c1);
            // one accumulator per spin component: four short dependency chains
            // of two-float additions instead of one of twelve
            df ax[4] = {df(0), df(0), df(0), df(0)}, ay[4] = {df(0), df(0), df(0), df(0)};
            const dfc* __restrict__ prv = side == 0 ? ring_q(o, rhs, jp) : ring_p(o, rhs, jp);
            dfc* __restrict__ nxt = side == 0 ? ring_q(o, rhs, j + 1) : ring_p(o, rhs, j + 1);
            const dfc* __restrict__ dotv = TS ? ring_p(o, rhs, j) : ring_q(o, rhs, j);
            double2* __restrict__ yacc = PASS2 ? o.y + (size_t)rhs * o.N : nullptr;
            const double2 cpj = PASS2 ? o.cp[hb + j] : make_double2(0.0, 0.0);
            const double2* __restrict__ qj = outer_q(o, rhs, j);
            for_each_out([&](int sp, int a, const T& vout) {
                const size_t idx = (size_t)(3 * sp + a) * g.V + site;
                const dfc v = to_dfc(vout);
                const dfc pv = prv[idx];
                dfc rr;
                if (TS || side == 1) {
                    rr.x = (v.x * scr.x - v.y * scr.y) - (c1d.x * pv.x - c1d.y * pv.y);   // s - c1 q_{j-1}
                    rr.y = (v.x * scr.y + v.y * scr.x) - (c1d.x * pv.y + c1d.y * pv.x);
                } else {
                    rr.x = v.x * scr.x - c1d.x * pv.x;
                    rr.y = v.y * scr.x - c1d.x * pv.y;
                }
                nxt[idx] = rr;
                if (side == 0) {
                    const dfc d = dotv[idx];
                    ax[sp] += d.x * rr.x + d.y * rr.y;        // conj(d) r
                    if (TS) ay[sp] += d.x * rr.y - d.y * rr.x;
                    if (PASS2) yacc[idx] = caxpy_pos(yacc[idx], cpj, qj[idx]);
                }
            });
            acc = make_double2(df_to_double((ax[0] + ax[1]) + (ax[2] + ax[3])),
                               df_to_double((ay[0] + ay[1]) + (ay[2] + ay[3])));
        }
        if (!ring_epilogue) {
            // the scale 1/n_j (1/m_j) in the stencil's precision
            T scr;
            scr.x = from_double<R>(coef[0].x);
            scr.y = from_double<R>(coef[0].y);
            if (side == 0) {
                const double2* __restrict__ prv = outer_q(o, rhs, jp);
                double2* __restrict__ nxt = outer_q(o, rhs, j + 1);   // at j = k-1 a scratch column
                const double2* __restrict__ dotv = TS ? outer_p(o, rhs, j) : outer_q(o, rhs, j);
                double2* __restrict__ yacc = PASS2 ? o.y + (size_t)rhs * o.N : nullptr;
                const double2 cpj = PASS2 ? o.cp[hb + j] : make_double2(0.0, 0.0);
                const double2* __restrict__ qj = outer_q(o, rhs, j);
                for_each_out([&](int sp, int a, const T& v) {
                    const size_t idx = (size_t)(3 * sp + a) * g.V + site;
                    double2 rr;
                    if (TS) {
                        rr = make_double2(to_double(v.x * scr.x - v.y * scr.y), to_double(v.x * scr.y + v.y * scr.x));
                        rr = caxpy_neg(rr, c1, prv[idx]);               // r - c1 q_{j-1}
                    } else {
                        rr = make_double2(to_double(v.x * scr.x), to_double(v.y * scr.x));
                        const double2 pv = prv[idx];
                        rr = make_double2(fma(-c1.x, pv.x, rr.x), fma(-c1.x, pv.y, rr.y));
                    }
                    nxt[idx] = rr;
                    const double2 d = dotv[idx];
                    acc.x = fma(d.x, rr.x, fma(d.y, rr.y, acc.x));          // conj(d) r
                    if (TS) acc.y = fma(d.x, rr.y, fma(-d.y, rr.x, acc.y));
                    if (PASS2) yacc[idx] = caxpy_pos(yacc[idx], cpj, qj[idx]);
                });
            } else {
                const double2* __restrict__ prv = outer_p(o, rhs, jp);
                double2* __restrict__ nxt = outer_p(o, rhs, j + 1);
                for_each_out([&](int sp, int a, const T& v) {
                    const size_t idx = (size_t)(3 * sp + a) * g.V + site;
                    double2 ll = make_double2(to_double(v.x * scr.x - v.y * scr.y), to_double(v.x * scr.y + v.y * scr.x));
                    nxt[idx] = caxpy_neg(ll, c1, prv[idx]);             // l - c1 p_{j-1}
                });
            }
        }
    }
    if (side == 0) {
        double2 part = block_sum(acc, sh);
        if (finish_partial(part, o.partials + (size_t)rhs * o.npart, o.counters + rhs, sb, nsb)) {
            double2 tot = sum_partials(o.partials + (size_t)rhs * o.npart, nsb, sh);
            // Hermitian: H(j,j) = Re(q_j^dag r) / n_j, real (App. C); two-sided: (p_j^dag r) / m_j^*;
            // with the step-2 scalars H(j,j)/n_j (warp 1) and H(j,j)^*/m_j (warp 0) side by side
            const int tid = block_tid();
            if (tid == 0 || tid == 32) {
                const double2 al = TS ? cmul(coef[2], tot) : make_double2(tot.x * coef[2].x, 0.0);
                if (tid == 0) {
                    o.alpha[hb + j] = al;
                    o.counters[rhs] = 0u;
                    o.sc[(size_t)rhs * kScalars + kScC4] = TS ? cdiv(cconj(al), scale_m(o, rhs, j))
                                                              : make_double2(0.0, 0.0);
                } else {
                    o.sc[(size_t)rhs * kScalars + kScC3] = cdiv(al, scale_n(o, rhs, j));
                }
            }
        }
    }
}

int dslash_step1_blocks(const Geom& g, int threads) { return (g.V + threads - 1) / threads; }

template <typename R, typename T, int CS>
static void launch_step1_cs(dim3 grid, dim3 block, const T* U, const Geom& g, const Outer& o, int j, R kappa,
                            R emu, R emu_inv, const T* qin, long qs, const T* pin, long ps, cudaStream_t st) {
    const bool pass2 = o.y != nullptr;
    if (o.two_sided) {
        if (pass2)
            k_dslash_step1<R, true, true, CS><<<grid, block, 0, st>>>(U, g, o, j, kappa, emu, emu_inv, qin, qs, pin, ps);
        else
            k_dslash_step1<R, true, false, CS><<<grid, block, 0, st>>>(U, g, o, j, kappa, emu, emu_inv, qin, qs, pin, ps);
    } else {
        if (pass2)
            k_dslash_step1<R, false, true, CS><<<grid, block, 0, st>>>(U, g, o, j, kappa, emu, emu_inv, qin, qs, pin, ps);
        else
            k_dslash_step1<R, false, false, CS><<<grid, block, 0, st>>>(U, g, o, j, kappa, emu, emu_inv, qin, qs, pin, ps);
    }
}

template <typename R, typename T>
static void launch_step1_t(const T* U, const Geom& g, const Outer& o, int j, R kappa, R emu, R emu_inv, const T* qin,
                           long qs, const T* pin, long ps, cudaStream_t st) {
    const int nvec = o.two_sided ? 2 * o.n_rhs : o.n_rhs;
    // launch shape of this precision (the kernel reads the grid order from o)
    Outer o2 = o;
    int split = o.st_split;
    if (std::is_same<R, df>::value) {
        o2.st_threads = o.st_threads_df;
        o2.st_order = o.st_order_df;
        split = o.st_split_df;
    }
    const int threads = o2.st_threads;
    dim3 grid((unsigned)(dslash_step1_blocks(g, threads) * nvec));
    if (split == 3)
        launch_step1_cs<R, T, 3>(grid, dim3(threads, 3), U, g, o2, j, kappa, emu, emu_inv, qin, qs, pin, ps, st);
    else
        launch_step1_cs<R, T, 1>(grid, dim3(threads, 1), U, g, o2, j, kappa, emu, emu_inv, qin, qs, pin, ps, st);
}

bool split_step(int precision, const Outer& o, int j) {
    return j < o.ring_from && ((precision == 32 && o.s32) || (precision == 48 && o.s64));
}

void launch_stencil_step(int precision, const void* U, const Geom& g, const Outer& o, int j, double kappa,
                         double mu, cudaStream_t st) {
    const int n_d = (o.two_sided && j < o.k - 1) ? o.n_rhs : 0;   // the last step needs no new left vector
    if (precision == 48) {
        StencilDfSet s;
        s.in_a = ring_q(o, 0, j);
        s.in_d = o.two_sided ? ring_p(o, 0, j) : nullptr;
        s.in_stride = 3 * o.N;   // rings [rhs][3][N]
        s.out_a = o.s64;
        s.out_d = o.s64 + (size_t)o.n_rhs * o.N;
        s.out_stride = o.N;
        s.n_a = o.n_rhs;
        s.n_d = n_d;
        s.scale = o.sc;
        launch_stencil_df(U, g, s, kappa, mu, st);
        return;
    }
    const long vs = o.N / 2;   // float4 per vector
    Stencil32Set s;
    s.in_a = o.q32;
    s.in_d = o.p32;
    s.out_a = o.s32;
    s.out_d = o.s32 + (size_t)o.n_rhs * vs;
    s.vstride = vs;
    s.n_a = o.n_rhs;
    s.n_d = n_d;
    s.scale = o.sc;
    launch_stencil32(U, g, s, kappa, mu, st);
}

int launch_dslash_step1(int precision, const void* U, const Geom& g, const Outer& o, int j, double kappa,
                        double mu, cudaStream_t st) {
    if (split_step(precision, o, j)) {
        // FP64 recurrence: the multi-RHS stencil leaves (A q_j)/n_j and
        // (A^dag p_j)/m_j in s32 / s64, a streaming FP64 kernel runs step 1 on them
        launch_stencil_step(precision, U, g, o, j, kappa, mu, st);
        launch_outer_step1(o, j, precision == 48, st);
        return 2;
    }
    if (precision == 32) {
        launch_stencil32_step1(U, g, o, j, kappa, mu, st);
    } else if (precision == 48) {   // the two-float stencil reads the two-float rings
        launch_step1_t<df, dfc>((const dfc*)U, g, o, j, df_host(kappa), df_host(exp(mu)), df_host(exp(-mu)),
                                ring_q(o, 0, j), 3 * o.N, o.two_sided ? ring_p(o, 0, j) : nullptr, 3 * o.N, st);
    } else {
        const long qs = (long)o.qcols * o.N;
        launch_step1_t<double, double2>((const double2*)U, g, o, j, kappa, exp(mu), exp(-mu), outer_q(o, 0, j), qs,
                                        o.two_sided ? outer_p(o, 0, j) : nullptr, (long)o.pcols * o.N, st);
    }
    return 1;
}

// ---- layout conversion -------------------------------------------------------

// ABI links [site][nu][3][3] complex double -> [nu][9][site] (FP64, FP32 and two-float copies)
__global__ void links_to_device_layout(const double2* __restrict__ in, double2* __restrict__ u64,
                                       float2* __restrict__ u32, dfc* __restrict__ udf, int V) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)V * 36) return;
    int site = (int)(i / 36), rem = (int)(i % 36), nu = rem / 9, e = rem % 9;
    double2 v = in[i];
    size_t o = (size_t)(nu * 9 + e) * V + site;
    u64[o] = v;
    u32[o] = make_float2((float)v.x, (float)v.y);
    dfc w;
    w.x = df_from_double(v.x);
    w.y = df_from_double(v.y);
    udf[o] = w;
}

void launch_links_to_device_layout(const double2* in, double2* u64, float2* u32, dfc* udf, int V,
                                   cudaStream_t st) {
    size_t n = (size_t)V * 36;
    links_to_device_layout<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, u64, u32, udf, V);
}

// ABI spinor [site][12] -> SoA [12][site], n vectors
__global__ void spinor_abi_to_soa(const double2* __restrict__ in, long in_stride, double2* __restrict__ out,
                                  long out_stride, int V, int n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t per = (size_t)V * 12;
    if (i >= per * n) return;
    int vec = (int)(i / per);
    size_t j = i % per;
    int site = (int)(j / 12), c = (int)(j % 12);
    out[(size_t)vec * out_stride + (size_t)c * V + site] = in[(size_t)vec * in_stride + j];
}

// SoA [12][site] -> ABI [site][12]; if add != nullptr: out = add + gamma5 * in (overlap)
__global__ void spinor_soa_to_abi(const double2* __restrict__ in, long in_stride, double2* __restrict__ out,
                                  long out_stride, const double2* __restrict__ add, long add_stride,
                                  int V, int n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t per = (size_t)V * 12;
    if (i >= per * n) return;
    int vec = (int)(i / per);
    size_t j = i % per;
    int site = (int)(j / 12), c = (int)(j % 12);
    double2 v = in[(size_t)vec * in_stride + (size_t)c * V + site];
    if (add) {
        double2 b = add[(size_t)vec * add_stride + j];
        double sg = c < 6 ? 1.0 : -1.0;  // gamma5 on spins 2, 3
        v = make_double2(b.x + sg * v.x, b.y + sg * v.y);
    }
    out[(size_t)vec * out_stride + j] = v;
}

void launch_abi_to_soa(const double2* in, long in_stride, double2* out, long out_stride, int V,
                       int n, cudaStream_t st) {
    size_t tot = (size_t)V * 12 * n;
    spinor_abi_to_soa<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(in, in_stride, out, out_stride,
                                                                      V, n);
}

void launch_soa_to_abi(const double2* in, long in_stride, double2* out, long out_stride,
                       const double2* add, long add_stride, int V, int n, cudaStream_t st) {
    size_t tot = (size_t)V * 12 * n;
    spinor_soa_to_abi<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(in, in_stride, out, out_stride,
                                                                      add, add_stride, V, n);
}

// ABI spinor [site][12] (double) -> FP32 pair layout [6][V] float4, n vectors
__global__ void abi_to_f32pair(const double2* __restrict__ in, long in_stride, float4* __restrict__ out,
                               long out_stride, int V, int n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // (vector, pair, site)
    const size_t per = (size_t)V * 6;
    if (i >= per * n) return;
    const int vec = (int)(i / per);
    const size_t rem = i % per;
    const int pr = (int)(rem / V), site = (int)(rem % V);
    const double2 a = in[(size_t)vec * in_stride + (size_t)site * 12 + 2 * pr];
    const double2 b = in[(size_t)vec * in_stride + (size_t)site * 12 + 2 * pr + 1];
    out[(size_t)vec * out_stride + rem] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

__global__ void f32pair_to_abi(const float4* __restrict__ in, long in_stride, double2* __restrict__ out,
                               long out_stride, int V, int n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t per = (size_t)V * 6;
    if (i >= per * n) return;
    const int vec = (int)(i / per);
    const size_t rem = i % per;
    const int pr = (int)(rem / V), site = (int)(rem % V);
    const float4 v = in[(size_t)vec * in_stride + rem];
    out[(size_t)vec * out_stride + (size_t)site * 12 + 2 * pr] = make_double2(v.x, v.y);
    out[(size_t)vec * out_stride + (size_t)site * 12 + 2 * pr + 1] = make_double2(v.z, v.w);
}

__global__ void to_df(const double2* __restrict__ in, long in_stride, dfc* __restrict__ out, long out_stride,
                      long N, int n) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)N * n) return;
    int vec = (int)(i / N);
    size_t j = i % N;
    double2 v = in[(size_t)vec * in_stride + j];
    dfc w;
    w.x = df_from_double(v.x);
    w.y = df_from_double(v.y);
    out[(size_t)vec * out_stride + j] = w;
}

void launch_to_df(const double2* in, long in_stride, dfc* out, long out_stride, long N, int n, cudaStream_t st) {
    size_t tot = (size_t)N * n;
    to_df<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(in, in_stride, out, out_stride, N, n);
}

void launch_abi_to_f32pair(const double2* in, long in_stride, float4* out, long out_stride, int V, int n,
                           cudaStream_t st) {
    const size_t tot = (size_t)V * 6 * n;
    abi_to_f32pair<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(in, in_stride, out, out_stride, V, n);
}

void launch_f32pair_to_abi(const float4* in, long in_stride, double2* out, long out_stride, int V, int n,
                           cudaStream_t st) {
    const size_t tot = (size_t)V * 6 * n;
    f32pair_to_abi<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(in, in_stride, out, out_stride, V, n);
}

}  // namespace nk

namespace nk {

// ---- mean plaquette (predictor feature) ----------------------------------------
// (1/3) Re tr U_mu(x)^+ U_nu(x+mu)^+ U_mu(x+nu) U_nu(x), summed over the six
// planes mu < nu of each site; one partial sum per block.  In the hop
// convention of Sec. 2 the link U_{x,+nu} transforms as W(x+nu) U W(x)^+, so
// this is the gauge-invariant closed loop.
// c = op(a) op(b), op = identity or conjugate transpose
__device__ __forceinline__ void su3_mul(const double2 a[3][3], bool adag, const double2 b[3][3], bool bdag,
                                        double2 c[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double2 s = make_double2(0.0, 0.0);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                const double2 x = adag ? make_double2(a[l][i].x, -a[l][i].y) : a[i][l];
                const double2 y = bdag ? make_double2(b[j][l].x, -b[j][l].y) : b[l][j];
                s.x += x.x * y.x - x.y * y.y;
                s.y += x.x * y.y + x.y * y.x;
            }
            c[i][j] = s;
        }
}

__global__ void k_plaquette(const double2* __restrict__ U, Geom g, double* __restrict__ partial) {
    __shared__ double sh[33];
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (site < g.V) {
        const int L[4] = {g.Lx, g.Ly, g.Lz, g.Lt};
        const int stride[4] = {1, g.Lx, g.Lx * g.Ly, g.Lx * g.Ly * g.Lz};
        int c[4];
        int r = site;
        for (int d = 0; d < 4; ++d) { c[d] = r % L[d]; r /= L[d]; }
        for (int mu = 0; mu < 4; ++mu) {
            const int xmu = c[mu] == L[mu] - 1 ? site - (L[mu] - 1) * stride[mu] : site + stride[mu];
            for (int nu = mu + 1; nu < 4; ++nu) {
                const int xnu = c[nu] == L[nu] - 1 ? site - (L[nu] - 1) * stride[nu] : site + stride[nu];
                double2 A[3][3], B[3][3], C[3][3], D[3][3], T1[3][3], T2[3][3];
                for (int e = 0; e < 9; ++e) {
                    A[e / 3][e % 3] = U[(size_t)(mu * 9 + e) * g.V + site];
                    B[e / 3][e % 3] = U[(size_t)(nu * 9 + e) * g.V + xmu];
                    C[e / 3][e % 3] = U[(size_t)(mu * 9 + e) * g.V + xnu];
                    D[e / 3][e % 3] = U[(size_t)(nu * 9 + e) * g.V + site];
                }
                su3_mul(A, true, B, true, T1);
                su3_mul(T1, false, C, false, T2);
                su3_mul(T2, false, D, false, T1);
                acc += (T1[0][0].x + T1[1][1].x + T1[2][2].x) / 3.0;
            }
        }
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

int plaquette_blocks(const Geom& g) { return (g.V + 127) / 128; }

void launch_plaquette(const double2* U, const Geom& g, double* partial, cudaStream_t st) {
    k_plaquette<<<plaquette_blocks(g), 128, 0, st>>>(U, g, partial);
}

}  // namespace nk
