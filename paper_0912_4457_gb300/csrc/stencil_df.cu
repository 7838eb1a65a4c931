// Multi-RHS two-float (about 48-bit) Wilson stencil A = gamma5 D_w(mu),
// A^dagger = gamma5 D_w(-mu) (Sec. 2): the stencil of the early outer steps of
// the mixed schedule, where an FP32 stencil would cost accuracy the later
// steps cannot recover.
//
// One CTA owns a block of kDfSites consecutive sites for every vector of the
// launch (threadIdx.x = site in the block, threadIdx.y = vector).  Before any
// vector is touched the CTA stages, in shared memory, the links of its sites'
// eight hops in the form the arithmetic uses -- M = U(x - nu) for the backward
// hops, M = U(x)^dagger for the forward ones, each element's real and
// imaginary part as broadcast pairs (hi, hi) and (lo, lo) -- with the
// neighbour indices and the boundary signs; every vector then reuses them.
//
// The arithmetic is two-float (a value is hi + lo, about 48 significant
// bits: TwoSum and TwoProd on the FP32 pipe) in the packed two-lane FP32
// instructions of sm_100+ (nk_f32x2.cuh): the two lanes carry the two
// half-spinor columns of a hop, which multiply the same link element, so one
// instruction serves both.  Per colour b a spinor is held as UR = (psi_0.re,
// psi_1.re), UI = (psi_0.im, psi_1.im), DR, DI (spins 2, 3).
//
// Input: two-float vectors (dfc, [vector][12][V]); output: FP64 vectors
// ([vector][12][V]) of gamma5 (psi - kappa hops), optionally scaled by the
// step scalar 1/n_j (A) or 1/m_j (A^dagger) in two-float arithmetic -- the
// input of the FP64 step-1 kernel.
#include "nk_common.cuh"
#include "nk_f32x2.cuh"
#include "nk_kernels.h"

namespace nk {

namespace {

constexpr int kDfSites = 8;                        // sites per CTA
constexpr int kDfMaxThreads = kDfSites * 24;   // 12 RHS of A and 12 of A^dagger

struct DfSmem {
    ulonglong2* lk;   // [((h * 9 + e) * 2 + part) * kDfSites + s]: part 0 re, 1 im, as {(hi, hi), (lo, lo)}
    int* nb;          // [h * kDfSites + s]
    float* fl;        // [h * kDfSites + s]: -1 across the antiperiodic t boundary, else 1
};

constexpr size_t df_smem() { return (size_t)kDfSites * (8 * 9 * 2 * 16 + 8 * 4 + 8 * 4); }

__device__ __forceinline__ DfSmem df_carve(char* sm) {
    DfSmem r;
    r.lk = reinterpret_cast<ulonglong2*>(sm);
    r.nb = reinterpret_cast<int*>(sm + (size_t)kDfSites * 8 * 9 * 2 * 16);
    r.fl = reinterpret_cast<float*>(sm + (size_t)kDfSites * (8 * 9 * 2 * 16 + 8 * 4));
    return r;
}

// Neighbour indices, boundary signs and the hop matrices of the CTA's sites
// (hop h: nu = h / 2, odd h forward).  Sites past V use site V - 1.
__device__ __forceinline__ void df_stage(const dfc* __restrict__ U, const Geom& g, int site0, const DfSmem& S) {
    const int tx = threadIdx.x, ty = threadIdx.y, vg = blockDim.y;
    const int site = min(site0 + tx, g.V - 1);
    if (ty == 0) {
        const int L[4] = {g.Lx, g.Ly, g.Lz, g.Lt};
        const int stride[4] = {1, g.Lx, g.Lx * g.Ly, g.Lx * g.Ly * g.Lz};
        int c[4];
        int r = site;
#pragma unroll
        for (int d = 0; d < 4; ++d) { c[d] = r % L[d]; r /= L[d]; }
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int nu = h >> 1;
            const bool fwd = (h & 1) != 0;
            const bool wrap = fwd ? c[nu] == L[nu] - 1 : c[nu] == 0;
            const int sn = fwd ? (wrap ? site - (L[nu] - 1) * stride[nu] : site + stride[nu])
                               : (wrap ? site + (L[nu] - 1) * stride[nu] : site - stride[nu]);
            S.nb[h * kDfSites + tx] = sn;
            S.fl[h * kDfSites + tx] = (nu == 3 && g.antiperiodic && wrap) ? -1.0f : 1.0f;
        }
    }
    __syncthreads();
    for (int q = ty; q < 72; q += vg) {
        const int h = q / 9, e = q % 9, nu = h >> 1, a = e / 3, b = e % 3;
        const bool fwd = (h & 1) != 0;
        // M_ab = U(x - nu)_ab backward, conj(U(x)_ba) forward
        const dfc u = fwd ? U[(size_t)(nu * 9 + 3 * b + a) * g.V + site]
                          : U[(size_t)(nu * 9 + e) * g.V + S.nb[h * kDfSites + tx]];
        const float ih = fwd ? -u.y.hi : u.y.hi, il = fwd ? -u.y.lo : u.y.lo;
        S.lk[(q * 2 + 0) * kDfSites + tx] = make_ulonglong2(pk(u.x.hi, u.x.hi), pk(u.x.lo, u.x.lo));
        S.lk[(q * 2 + 1) * kDfSites + tx] = make_ulonglong2(pk(ih, ih), pk(il, il));
    }
    __syncthreads();
}

struct DSpin {
    P2 ur[3], ui[3], dr[3], di[3];
};

// the two-float spinor of site s (components 3 sp + b, each (re.hi, re.lo,
// im.hi, im.lo)) in the spin-pair lanes
__device__ __forceinline__ void load_dspin(const dfc* __restrict__ in, int V, int s, DSpin& p) {
    const float4* f = reinterpret_cast<const float4*>(in);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const float4 s0 = __ldg(f + (size_t)b * V + s), s1 = __ldg(f + (size_t)(3 + b) * V + s);
        const float4 s2 = __ldg(f + (size_t)(6 + b) * V + s), s3 = __ldg(f + (size_t)(9 + b) * V + s);
        p.ur[b] = {pk(s0.x, s1.x), pk(s0.y, s1.y)};
        p.ui[b] = {pk(s0.z, s1.z), pk(s0.w, s1.w)};
        p.dr[b] = {pk(s2.x, s3.x), pk(s2.y, s3.y)};
        p.di[b] = {pk(s2.z, s3.z), pk(s2.w, s3.w)};
    }
}

// lane signs (S0, S1) in {+1, -1} times the hop sign s (forward hops: -1),
// exact: m is the sign-bit mask of s in both lanes
template <int S0, int S1>
__device__ __forceinline__ P2 sgn(P2 a, f2p m) {
    constexpr f2p k = (S0 < 0 ? 0x0000000080000000ull : 0ull) | (S1 < 0 ? 0x8000000000000000ull : 0ull);
    return {a.s ^ m ^ k, a.e ^ m ^ k};
}

// One hop into the accumulators: acc += w (1 + s gamma_nu) M psi_n with
// s = +1 backward (M = U(x - nu)), -1 forward (M = U(x)^dagger), in the
// chiral basis:
//   (C psi_dn)_{0,1}:  nu = x: -i psi_3, -i psi_2;  y: -psi_3, psi_2;
//                      z: -i psi_2, i psi_3;       t: psi_2, psi_3
//   (B m)_{0,1}:       nu = x: i m_1, i m_0;        y: m_1, -m_0;
//                      z: i m_0, -i m_1;           t: m_0, m_1
// (i z = (-z.im, z.re)); the spin swaps of x and y become swaps of the lanes.
// One instantiation per direction; the forward and backward hops of it share
// the code (fwd a runtime value), which halves the kernel's instruction
// footprint -- the fully unrolled eight hops overflowed the instruction cache.
template <int NU>
__device__ __forceinline__ void df_hop(DSpin& acc, const dfc* __restrict__ in, int V, const DfSmem& S, df wp_t,
                                       df wm_t, int fwd) {
    constexpr int SG = 1;   // lane signs below are for the backward hop; m flips them forward
    const int H = 2 * NU + fwd;
    const f2p m = fwd ? 0x8000000080000000ull : 0ull;
    const int tx = threadIdx.x;
    DSpin p;
    load_dspin(in, V, S.nb[H * kDfSites + tx], p);
    // projection: HR = (h0.re, h1.re), HI = (h0.im, h1.im) per colour, and -HI
    P2 hr[3], hi[3], nhi[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (NU == 0) {        // c0 = -i psi3 = (psi3.im, -psi3.re), c1 = -i psi2
            hr[b] = p2_add(p.ur[b], sgn<SG, SG>(p2_swp(p.di[b]), m));
            hi[b] = p2_add(p.ui[b], sgn<-SG, -SG>(p2_swp(p.dr[b]), m));
        } else if (NU == 1) { // c0 = -psi3, c1 = psi2
            hr[b] = p2_add(p.ur[b], sgn<-SG, SG>(p2_swp(p.dr[b]), m));
            hi[b] = p2_add(p.ui[b], sgn<-SG, SG>(p2_swp(p.di[b]), m));
        } else if (NU == 2) { // c0 = -i psi2 = (psi2.im, -psi2.re), c1 = i psi3 = (-psi3.im, psi3.re)
            hr[b] = p2_add(p.ur[b], sgn<SG, -SG>(p.di[b], m));
            hi[b] = p2_add(p.ui[b], sgn<-SG, SG>(p.dr[b], m));
        } else {              // c0 = psi2, c1 = psi3
            hr[b] = p2_add(p.ur[b], sgn<SG, SG>(p.dr[b], m));
            hi[b] = p2_add(p.ui[b], sgn<SG, SG>(p.di[b], m));
        }
        nhi[b] = p2_neg(hi[b]);
    }
    P2 wt;   // the temporal weight e^{+-mu} with the boundary sign (t hops only)
    if (NU == 3) {
        const df w = fwd ? wm_t : wp_t;
        const float f = S.fl[H * kDfSites + tx];
        wt = {pk(w.hi * f, w.hi * f), pk(w.lo * f, w.lo * f)};
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        P2 xr, xi;   // (x0, x1) = row a of M times (h0, h1)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int q = H * 9 + 3 * a + b;
            const ulonglong2 mr2 = S.lk[(q * 2 + 0) * kDfSites + tx], mi2 = S.lk[(q * 2 + 1) * kDfSites + tx];
            const P2 mr = {mr2.x, mr2.y}, mi = {mi2.x, mi2.y};
            if (b == 0) {
                xr = p2_prod(mr, hr[b]);
                xi = p2_prod(mr, hi[b]);
            } else {
                p2_add_prod(xr, mr, hr[b]);
                p2_add_prod(xi, mr, hi[b]);
            }
            p2_add_prod(xr, mi, nhi[b]);   // re: mr hr - mi hi
            p2_add_prod(xi, mi, hr[b]);    // im: mr hi + mi hr
        }
        if (NU == 3) {
            xr = p2_prod(wt, xr);
            xi = p2_prod(wt, xi);
        }
        acc.ur[a] = p2_add(acc.ur[a], xr);
        acc.ui[a] = p2_add(acc.ui[a], xi);
        if (NU == 0) {        // b0 = i x1, b1 = i x0: (-x1.im, -x0.im), (x1.re, x0.re)
            acc.dr[a] = p2_add(acc.dr[a], sgn<-SG, -SG>(p2_swp(xi), m));
            acc.di[a] = p2_add(acc.di[a], sgn<SG, SG>(p2_swp(xr), m));
        } else if (NU == 1) { // b0 = x1, b1 = -x0
            acc.dr[a] = p2_add(acc.dr[a], sgn<SG, -SG>(p2_swp(xr), m));
            acc.di[a] = p2_add(acc.di[a], sgn<SG, -SG>(p2_swp(xi), m));
        } else if (NU == 2) { // b0 = i x0 = (-x0.im, x0.re), b1 = -i x1 = (x1.im, -x1.re)
            acc.dr[a] = p2_add(acc.dr[a], sgn<-SG, SG>(xi, m));
            acc.di[a] = p2_add(acc.di[a], sgn<SG, -SG>(xr, m));
        } else {              // b0 = x0, b1 = x1
            acc.dr[a] = p2_add(acc.dr[a], sgn<SG, SG>(xr, m));
            acc.di[a] = p2_add(acc.di[a], sgn<SG, SG>(xi, m));
        }
    }
}

// two lanes of a two-float pair as FP64 (integer-pipe conversions, one FP64 add)
__device__ __forceinline__ void p2_to_double(P2 v, double& l0, double& l1) {
    float s0, s1, e0, e1;
    upk(v.s, s0, s1);
    upk(v.e, e0, e1);
    l0 = f2d_int(s0) + f2d_int(e0);
    l1 = f2d_int(s1) + f2d_int(e1);
}

__global__ void __launch_bounds__(kDfMaxThreads, 2) k_stencil_df(const dfc* __restrict__ U, Geom g, StencilDfSet s,
                                                              df kappa, df emu, df emu_inv) {
    extern __shared__ __align__(16) char smem[];
    const DfSmem S = df_carve(smem);
    const int site0 = blockIdx.x * kDfSites;
    const int site = min(site0 + (int)threadIdx.x, g.V - 1);
    df_stage(U, g, site0, S);
    const int v = threadIdx.y;
    if (v >= s.n_a + s.n_d) return;
    const int side = v < s.n_a ? 0 : 1;
    const int vi = side ? v - s.n_a : v;
    const dfc* __restrict__ in = (side ? s.in_d : s.in_a) + (size_t)vi * s.in_stride;
    // temporal weights: A uses (e^{mu}, e^{-mu}); A^dagger exchanges them
    const df wp_t = side ? emu_inv : emu, wm_t = side ? emu : emu_inv;
    DSpin acc;
#pragma unroll
    for (int a = 0; a < 3; ++a) acc.ur[a] = acc.ui[a] = acc.dr[a] = acc.di[a] = P2{0ull, 0ull};
#pragma unroll 1
    for (int f = 0; f < 2; ++f) df_hop<0>(acc, in, g.V, S, wp_t, wm_t, f);
#pragma unroll 1
    for (int f = 0; f < 2; ++f) df_hop<1>(acc, in, g.V, S, wp_t, wm_t, f);
#pragma unroll 1
    for (int f = 0; f < 2; ++f) df_hop<2>(acc, in, g.V, S, wp_t, wm_t, f);
#pragma unroll 1
    for (int f = 0; f < 2; ++f) df_hop<3>(acc, in, g.V, S, wp_t, wm_t, f);
    if (site0 + (int)threadIdx.x >= g.V) return;
    DSpin p;
    load_dspin(in, g.V, site, p);
    const P2 K = {pk(kappa.hi, kappa.hi), pk(kappa.lo, kappa.lo)};
    P2 SR, SI;   // the scale 1/n_j (1/m_j), two-float from its FP64 value
    const bool scaled = s.scale != nullptr;
    if (scaled) {
        const double2 z = s.scale[(size_t)vi * kScalars + (side ? kScM : kScN)];
        const df zr = df_from_double(z.x), zi = df_from_double(z.y);
        SR = {pk(zr.hi, zr.hi), pk(zr.lo, zr.lo)};
        SI = {pk(zi.hi, zi.hi), pk(zi.lo, zi.lo)};
    }
    double2* __restrict__ out = (side ? s.out_d : s.out_a) + (size_t)vi * s.out_stride;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // gamma5 = diag(1, 1, -1, -1): upper spins psi - kappa acc, lower kappa acc - psi
        P2 yr[2], yi[2];
        yr[0] = p2_add(p.ur[a], p2_neg(p2_prod(K, acc.ur[a])));
        yi[0] = p2_add(p.ui[a], p2_neg(p2_prod(K, acc.ui[a])));
        yr[1] = p2_add(p2_prod(K, acc.dr[a]), p2_neg(p.dr[a]));
        yi[1] = p2_add(p2_prod(K, acc.di[a]), p2_neg(p.di[a]));
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            P2 orr = yr[hf], oii = yi[hf];
            if (scaled) {   // (yr + i yi)(sr + i si)
                orr = p2_add(p2_prod(SR, yr[hf]), p2_prod(SI, p2_neg(yi[hf])));
                oii = p2_add(p2_prod(SI, yr[hf]), p2_prod(SR, yi[hf]));
            }
            double r0, r1, i0, i1;
            p2_to_double(orr, r0, r1);
            p2_to_double(oii, i0, i1);
            out[(size_t)(3 * (2 * hf) + a) * g.V + site] = make_double2(r0, i0);
            out[(size_t)(3 * (2 * hf + 1) + a) * g.V + site] = make_double2(r1, i1);
        }
    }
}

df df_of_host(double d) {
    df r;
    r.hi = (float)d;
    r.lo = (float)(d - (double)r.hi);
    return r;
}

}  // namespace

void stencil_df_init_attributes() {
    cudaFuncSetAttribute(k_stencil_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)df_smem());
}

void launch_stencil_df(const void* Udf, const Geom& g, const StencilDfSet& s, double kappa, double mu,
                       cudaStream_t st) {
    const int nv = s.n_a + s.n_d;
    if (nv == 0) return;
    const dim3 block(kDfSites, nv);
    const unsigned grid = (unsigned)((g.V + kDfSites - 1) / kDfSites);
    k_stencil_df<<<grid, block, df_smem(), st>>>((const dfc*)Udf, g, s, df_of_host(kappa), df_of_host(exp(mu)),
                                                  df_of_host(exp(-mu)));
}

}  // namespace nk
