// Multi-RHS FP32 Wilson stencil A = gamma5 D_w(mu), A^dagger = gamma5 D_w(-mu)
// (Sec. 2), the stencil of the late outer steps of the mixed schedule.
//
// One CTA owns a block of SB consecutive lattice sites for every vector of the
// launch (up to 12 right-hand sides of A and 12 of A^dagger; threadIdx.x = site
// in the block, threadIdx.y = vector slot, looping over vectors in groups of
// blockDim.y).  Before any vector is touched the CTA stages, in shared memory,
// the eight links its sites' hops use -- U_nu(x) for the forward hops (applied
// as U^dagger) and U_nu(x - nu) for the backward ones -- together with the
// neighbour indices and the boundary signs, so each link is read from global
// memory once per CTA and then applied to all vectors (the RHS of the batch
// and both sides of the two-sided recurrence share the operator).
//
// FP32 vectors use the pair layout [vector][6][V] of float4: float4 i of a site
// holds spin-colour components 2i and 2i + 1 (component = 3 spin + colour), so
// a neighbour spinor is six 16-byte loads, each coalesced over the sites of a
// warp.  The links stay [nu][9][V] float2 in global memory; in shared memory
// each hop's nine elements are five float4 (the tenth element is padding).
//
// Two kernels share the site loop: k_stencil32 stores FP32 outputs (the
// stencil alone, nk_stencil32_dev and nk_dslash_dev, and the stencil of the
// FP32 steps of an FP64 recurrence, whose step 1 then runs as a streaming
// FP64 kernel in lanczos.cu), k_stencil32_step1 runs the first half of outer
// step j of the optional two-float recurrence on the output (lanczos.cu
// describes the unnormalised basis):
//   side 0: r = (A q_j) / n_j - (c_{j-1}/n_{j-1}) q_{j-1} -> q_{j+1},
//           H(j,j) = (p_j^dag r) / m_j^*  (Hermitian: Re(q_j^dag r) / n_j),
//   side 1: l = (A^dag p_j) / m_j - (beta^*_{j-1}/m_{j-1}) p_{j-1} -> p_{j+1},
// with the stencil output and its scale 1/n_j in FP32 (the stencil
// application) and the update, the inner product and its accumulation in
// FP64 on the FP64 vectors; or, from step ring_from on (the optional
// two-float recurrence), in two-float arithmetic on the rings.  H(j,j) is
// reduced deterministically: a fixed-order sum over the sites of each CTA,
// one partial per CTA and RHS, and a fixed-order sum of the partials in the
// CTA that finishes last (integer ticket), which also forms the step-2
// scalars of the step.
#include "nk_common.cuh"
#include "nk_hop.cuh"
#include "nk_kernels.h"

namespace nk {

namespace {

// Shared memory of a CTA of sb sites: links (8 hops x 5 float4 per site),
// neighbour site and boundary sign per hop.  (A variant that also prefetched
// each thread's next neighbour spinor into shared memory with cp.async was
// slower: the spinors then cross the L1/shared-memory datapath twice, which
// ran at 92% of its throughput, and lost their L1 hits.)
__host__ __device__ constexpr size_t s32_smem(int sb, int nth) {
    return (void)nth, (size_t)sb * (8 * 5 * 16 + 8 * 4 + 8 * 4);
}

struct S32Smem {
    float4* lk;   // [(h * 5 + q) * SB + s]
    int* nb;      // [h * SB + s]
    float* fl;    // [h * SB + s]: -1 across the antiperiodic t boundary, else 1
};

__device__ __forceinline__ S32Smem s32_carve(char* sm, int sb) {
    S32Smem r;
    r.lk = reinterpret_cast<float4*>(sm);
    r.nb = reinterpret_cast<int*>(sm + (size_t)sb * 8 * 5 * 16);
    r.fl = reinterpret_cast<float*>(sm + (size_t)sb * (8 * 5 * 16 + 8 * 4));
    return r;
}

// Asynchronous global -> shared copies (cp.async) for the link staging: the
// copies of one thread form a group, and wait_group 0 returns once they have
// all landed.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void load_spinor32(const float4* __restrict__ in, int V, int s, float2 p[4][3]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float4 v = __ldg(in + (size_t)i * V + s);
        const int c0 = 2 * i, c1 = 2 * i + 1;
        p[c0 / 3][c0 % 3] = make_float2(v.x, v.y);
        p[c1 / 3][c1 % 3] = make_float2(v.z, v.w);
    }
}

// Neighbour indices and boundary signs of the CTA's sites (hop h: nu = h / 2,
// odd h forward), then the asynchronous copies of their links into shared
// memory as one group (waited for by s32_stage_end).  Sites past V (the last block)
// use site V - 1 and are skipped later.
__device__ __forceinline__ void s32_stage_begin(const float2* __restrict__ U, const Geom& g, int site0,
                                                const S32Smem& S) {
    const int sb = blockDim.x, tx = threadIdx.x, ty = threadIdx.y, vg = blockDim.y;
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
            S.nb[h * sb + tx] = sn;
            S.fl[h * sb + tx] = (nu == 3 && g.antiperiodic && wrap) ? -1.0f : 1.0f;
        }
    }
    __syncthreads();
    for (int q = ty; q < 40; q += vg) {
        const int h = q / 5, pr = q % 5, nu = h >> 1;
        const int ls = (h & 1) ? site : S.nb[h * sb + tx];
        float4* dst = S.lk + q * sb + tx;
        cp_async8(dst, U + (size_t)(nu * 9 + 2 * pr) * g.V + ls);
        if (pr < 4) cp_async8(reinterpret_cast<float2*>(dst) + 1, U + (size_t)(nu * 9 + 2 * pr + 1) * g.V + ls);
    }
    cp_async_commit();
}

// Wait for this thread's link copies, then for everyone's.
__device__ __forceinline__ void s32_stage_end() {
    cp_async_wait_all();
    __syncthreads();
}

// One hop: the neighbour spinor straight from global memory (L1 / L2), the
// link from shared memory.
template <int H>
__device__ __forceinline__ void s32_hop(float2 acc[4][3], const float4* __restrict__ in, int V, const S32Smem& S,
                                        float wp_t, float wm_t) {
    constexpr int NU = H >> 1;
    constexpr bool FWD = (H & 1) != 0;
    const int sb = blockDim.x, tx = threadIdx.x;
    float2 psi[4][3];
    load_spinor32(in, V, S.nb[H * sb + tx], psi);
    float2 u[3][3];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const float4 v = S.lk[(H * 5 + q) * sb + tx];
        const int e0 = 2 * q, e1 = 2 * q + 1;
        u[e0 / 3][e0 % 3] = make_float2(v.x, v.y);
        if (e1 < 9) u[e1 / 3][e1 % 3] = make_float2(v.z, v.w);
    }
    const float w = (NU == 3 ? (FWD ? wm_t : wp_t) : 1.0f) * S.fl[H * sb + tx];
    hop_regs<NU, FWD, float>(acc, psi, u, FWD ? -1.0f : 1.0f, w);
}

// out = gamma5 (psi - kappa * sum of the eight hops) at this thread's site
// (clamped to the lattice), for the vector `in`; side 1 (A^dagger) exchanges
// the temporal weights.
__device__ __forceinline__ void s32_site(const float4* __restrict__ in, int V, int site, const S32Smem& S, int side,
                                         float kappa, float emu, float emu_inv, float2 out[4][3]) {
    const float wp_t = side ? emu_inv : emu;
    const float wm_t = side ? emu : emu_inv;
    float2 acc[4][3];
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[sp][a] = make_float2(0.f, 0.f);
    s32_hop<0>(acc, in, V, S, wp_t, wm_t);
    s32_hop<1>(acc, in, V, S, wp_t, wm_t);
    s32_hop<2>(acc, in, V, S, wp_t, wm_t);
    s32_hop<3>(acc, in, V, S, wp_t, wm_t);
    s32_hop<4>(acc, in, V, S, wp_t, wm_t);
    s32_hop<5>(acc, in, V, S, wp_t, wm_t);
    s32_hop<6>(acc, in, V, S, wp_t, wm_t);
    s32_hop<7>(acc, in, V, S, wp_t, wm_t);
    float2 p[4][3];
    load_spinor32(in, V, site, p);
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
        const float sg = sp < 2 ? 1.0f : -1.0f;   // gamma5 = diag(1, 1, -1, -1)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            out[sp][a] = make_float2(sg * (p[sp][a].x - kappa * acc[sp][a].x), sg * (p[sp][a].y - kappa * acc[sp][a].y));
    }
}

// ---- the stencil alone: FP32 in, FP32 out ---------------------------------------
__global__ void __launch_bounds__(384, 2) k_stencil32(const float2* __restrict__ U, Geom g, Stencil32Set s, float kappa,
                                                      float emu, float emu_inv) {
    extern __shared__ __align__(16) char smem[];
    const S32Smem S = s32_carve(smem, blockDim.x);
    const int site0 = blockIdx.x * blockDim.x;
    const int site = min(site0 + (int)threadIdx.x, g.V - 1);
    const int nv = s.n_a + s.n_d;
    auto vec_in = [&](int v) {
        const int side = v < s.n_a ? 0 : 1;
        return (side ? s.in_d : s.in_a) + (size_t)(side ? v - s.n_a : v) * s.vstride;
    };
    s32_stage_begin(U, g, site0, S);
    s32_stage_end();
    for (int v = threadIdx.y; v < nv; v += blockDim.y) {
        const int side = v < s.n_a ? 0 : 1;
        const int vi = side ? v - s.n_a : v;
        float2 o[4][3];
        s32_site(vec_in(v), g.V, site, S, side, kappa, emu, emu_inv, o);
        if (site0 + (int)threadIdx.x >= g.V) continue;
        if (s.scale) {   // A v_j = (A q_j) / n_j (A^dagger w_j = (A^dagger p_j) / m_j), in FP32
            const double2 z = s.scale[(size_t)vi * kScalars + (side ? kScM : kScN)];
            const float2 f = make_float2(d2f_int(z.x), d2f_int(z.y));
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float2 w = o[sp][a];
                    o[sp][a] = make_float2(w.x * f.x - w.y * f.y, w.x * f.y + w.y * f.x);
                }
        }
        float4* out = (side ? s.out_d : s.out_a) + (size_t)vi * s.vstride;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const int c0 = 2 * i, c1 = 2 * i + 1;
            const float2 a = o[c0 / 3][c0 % 3], b = o[c1 / 3][c1 % 3];
            out[(size_t)i * g.V + site] = make_float4(a.x, a.y, b.x, b.y);
        }
    }
}

// two-float complex from an FP32 stencil output or a double (integer-pipe
// conversion, see nk_common.cuh)
__device__ __forceinline__ dfc dfc_f(float2 v) {
    dfc r;
    r.x = df(v.x, 0.0f);
    r.y = df(v.y, 0.0f);
    return r;
}
__device__ __forceinline__ dfc dfc_d(double2 v) {
    dfc r;
    r.x = df_from_double(v.x);
    r.y = df_from_double(v.y);
    return r;
}
__device__ __forceinline__ double2 cfma_neg(double2 s, double2 c, double2 p) {   // s - c p
    return make_double2(fma(-c.x, p.x, fma(c.y, p.y, s.x)), fma(-c.x, p.y, fma(-c.y, p.x, s.y)));
}
__device__ __forceinline__ double2 cfma_pos(double2 s, double2 c, double2 p) {   // s + c p
    return make_double2(fma(c.x, p.x, fma(-c.y, p.y, s.x)), fma(c.x, p.y, fma(c.y, p.x, s.y)));
}

// ---- fused with the first half of outer step j ------------------------------------
// RING: the two-float recurrence (j >= o.ring_from).  Shared memory after the
// stencil's: the per-(vector slot) H(j,j) partial sums of the CTA.
template <bool TS, bool PASS2, bool RING>
__global__ void __launch_bounds__(384, 2) k_stencil32_step1(const float2* __restrict__ U, Geom g, Outer o, int j,
                                                         float kappa, float emu, float emu_inv) {
    extern __shared__ __align__(16) char smem[];
    __shared__ bool last;
    const int sb = blockDim.x;
    const S32Smem S = s32_carve(smem, sb);
    const int site0 = blockIdx.x * sb;
    const int site = min(site0 + (int)threadIdx.x, g.V - 1);
    const bool live = site0 + (int)threadIdx.x < g.V;
    const int nrhs = o.n_rhs;
    const int nv = TS ? 2 * nrhs : nrhs;
    const int V = g.V;
    auto vec_in = [&](int v) {
        return (v < nrhs ? o.q32 + (size_t)v * 6 * V : o.p32 + (size_t)(v - nrhs) * 6 * V);
    };
    s32_stage_begin(U, g, site0, S);
    s32_stage_end();
    const int nblk = gridDim.x;
    const int tid = threadIdx.x + sb * threadIdx.y;   // linear: a warp may span two slots (sb = 16)
    const int lane = tid & 31;
    // every thread runs the same number of passes (the shuffles below need the
    // whole warp); a slot without a live vector contributes zero
    for (int base = 0; base < nv; base += blockDim.y) {
        const int v = base + threadIdx.y;
        const int side = v < nrhs ? 0 : 1;
        const int rhs = v < nv ? (side ? v - nrhs : v) : 0;
        const bool work = v < nv && o.status[rhs] == kStatusOK && !(side == 1 && j == o.k - 1);
        double2 acc = make_double2(0.0, 0.0);
        if (work) {
            const double2* sc = o.sc + (size_t)rhs * kScalars;
            const size_t hb = (size_t)rhs * o.k;
            const int jp = j > 0 ? j - 1 : j;
            float2 out[4][3];
            s32_site(vec_in(v), V, site, S, side, kappa, emu, emu_inv, out);
            if (live) {
            const double2 s0 = sc[side ? kScM : kScN];       // 1/n_j (1/m_j)
            const double2 c1 = sc[side ? kScC1L : kScC1];    // zero at j = 0
            const float2 scr = make_float2(d2f_int(s0.x), d2f_int(s0.y));
            if (!RING) {
                const double2* __restrict__ prv = side ? outer_p(o, rhs, jp) : outer_q(o, rhs, jp);
                double2* __restrict__ nxt = side ? outer_p(o, rhs, j + 1) : outer_q(o, rhs, j + 1);
                const double2* __restrict__ dotv = TS ? outer_p(o, rhs, j) : outer_q(o, rhs, j);
                double2* __restrict__ yacc = PASS2 ? o.y + (size_t)rhs * o.N : nullptr;
                const double2 cpj = PASS2 ? o.cp[hb + j] : make_double2(0.0, 0.0);
                const double2* __restrict__ qj = outer_q(o, rhs, j);
#pragma unroll
                for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const size_t idx = (size_t)(3 * sp + a) * V + site;
                        const float2 vo = out[sp][a];
                        // the stencil output times its scale, in FP32 (the stencil application)
                        double2 rr;
                        if (TS || side) rr = make_double2(f2d_int(vo.x * scr.x - vo.y * scr.y),
                                                          f2d_int(vo.x * scr.y + vo.y * scr.x));
                        else rr = make_double2(f2d_int(vo.x * scr.x), f2d_int(vo.y * scr.x));
                        if (TS || side) rr = cfma_neg(rr, c1, prv[idx]);
                        else {
                            const double2 pv = prv[idx];
                            rr = make_double2(fma(-c1.x, pv.x, rr.x), fma(-c1.x, pv.y, rr.y));
                        }
                        nxt[idx] = rr;
                        if (!side) {
                            const double2 d = dotv[idx];
                            acc.x = fma(d.x, rr.x, fma(d.y, rr.y, acc.x));      // conj(d) r
                            if (TS) acc.y = fma(d.x, rr.y, fma(-d.y, rr.x, acc.y));
                            if (PASS2) yacc[idx] = cfma_pos(yacc[idx], cpj, qj[idx]);
                        }
                    }
            } else {
                const dfc scd = dfc_d(s0), c1d = dfc_d(c1);
                const dfc* __restrict__ prv = side ? ring_p(o, rhs, jp) : ring_q(o, rhs, jp);
                dfc* __restrict__ nxt = side ? ring_p(o, rhs, j + 1) : ring_q(o, rhs, j + 1);
                const dfc* __restrict__ dotv = TS ? ring_p(o, rhs, j) : ring_q(o, rhs, j);
                double2* __restrict__ yacc = PASS2 ? o.y + (size_t)rhs * o.N : nullptr;
                const double2 cpj = PASS2 ? o.cp[hb + j] : make_double2(0.0, 0.0);
                const double2* __restrict__ qj = outer_q(o, rhs, j);
                df ax[4] = {df(0), df(0), df(0), df(0)}, ay[4] = {df(0), df(0), df(0), df(0)};
#pragma unroll
                for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const size_t idx = (size_t)(3 * sp + a) * V + site;
                        const dfc vv = dfc_f(out[sp][a]);
                        const dfc pv = prv[idx];
                        dfc rr;
                        if (TS || side) {
                            rr.x = (vv.x * scd.x - vv.y * scd.y) - (c1d.x * pv.x - c1d.y * pv.y);
                            rr.y = (vv.x * scd.y + vv.y * scd.x) - (c1d.x * pv.y + c1d.y * pv.x);
                        } else {
                            rr.x = vv.x * scd.x - c1d.x * pv.x;
                            rr.y = vv.y * scd.x - c1d.x * pv.y;
                        }
                        nxt[idx] = rr;
                        if (!side) {
                            const dfc d = dotv[idx];
                            ax[sp] += d.x * rr.x + d.y * rr.y;
                            if (TS) ay[sp] += d.x * rr.y - d.y * rr.x;
                            if (PASS2) yacc[idx] = cfma_pos(yacc[idx], cpj, qj[idx]);
                        }
                    }
                acc = make_double2(df_to_double((ax[0] + ax[1]) + (ax[2] + ax[3])),
                                   df_to_double((ay[0] + ay[1]) + (ay[2] + ay[3])));
            }
            }
        }
        // fixed-order sum over the sb sites of this vector slot: sb <= 32 lanes
        // of one warp (blockDim.x = sb, so a warp holds 32 / sb whole slots)
        double2 t = acc;
        for (int off = sb >> 1; off > 0; off >>= 1) {
            t.x += __shfl_xor_sync(0xffffffffu, t.x, off, sb);
            t.y += __shfl_xor_sync(0xffffffffu, t.y, off, sb);
        }
        if (v < nv && side == 0 && threadIdx.x == 0 && o.status[rhs] == kStatusOK)
            o.partials[(size_t)rhs * o.npart + blockIdx.x] = t;
    }
    // ticket: the CTA that finishes last sums every RHS's partials in a fixed order
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(o.counters, 1u);
        last = ticket == (unsigned)nblk - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int nthreads = sb * blockDim.y;
    const int w = tid >> 5, nw = nthreads >> 5;
    for (int rhs = w; rhs < nrhs; rhs += nw) {
        if (o.status[rhs] != kStatusOK) continue;
        double2 a = make_double2(0.0, 0.0);
        for (int i = lane; i < nblk; i += 32) {
            const double2 v = __ldcg(o.partials + (size_t)rhs * o.npart + i);
            a.x += v.x;
            a.y += v.y;
        }
        a = warp_sum(a);
        const double2* sc = o.sc + (size_t)rhs * kScalars;
        const size_t at = (size_t)rhs * o.k + j;
        // Hermitian: H(j,j) = Re(q_j^dag r) / n_j, real (App. C); two-sided: (p_j^dag r) / m_j^*
        const double2 al = TS ? cmul(sc[kScD], a) : make_double2(a.x * sc[kScD].x, 0.0);
        if (lane == 0) o.alpha[at] = al;
        // the step-2 scalars H(j,j)/n_j and H(j,j)^*/m_j, one per lane
        if (lane == 1) o.sc[(size_t)rhs * kScalars + kScC3] = cdiv(al, scale_n(o, rhs, j));
        if (lane == 2) o.sc[(size_t)rhs * kScalars + kScC4] = TS ? cdiv(cconj(al), scale_m(o, rhs, j))
                                                                 : make_double2(0.0, 0.0);
    }
    if (tid == 0) o.counters[0] = 0u;
}

}  // namespace

int stencil32_sites_per_cta(int nv) {
    // 8 sites for more than 12 vectors (192 threads for 24: more, smaller
    // CTAs in flight, measured 4% faster than 16 sites at 24 vectors), else
    // 32; at most 32, so that the sites of one vector slot sit in one warp,
    // and at most 384 threads, so that two CTAs (with their spinor slots) fit
    // an SM
    return nv > 12 ? 8 : 32;
}

int stencil32_blocks(const Geom& g, int nv) {
    const int sb = stencil32_sites_per_cta(nv);
    return (g.V + sb - 1) / sb;
}

static dim3 s32_block(int nv) {
    // sites x vector slots, one slot per vector (at most 32 x 12 or 8 x 24 threads)
    return dim3(stencil32_sites_per_cta(nv), nv);
}

void stencil32_init_attributes() {
    const int smax = (int)s32_smem(16, 384) > (int)s32_smem(32, 384) ? (int)s32_smem(16, 384) : (int)s32_smem(32, 384);
    cudaFuncSetAttribute(k_stencil32, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
#define NK_S1A(TS_, P2_, R_) \
    cudaFuncSetAttribute(k_stencil32_step1<TS_, P2_, R_>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax)
    NK_S1A(true, true, true); NK_S1A(true, true, false); NK_S1A(true, false, true); NK_S1A(true, false, false);
    NK_S1A(false, true, true); NK_S1A(false, true, false); NK_S1A(false, false, true); NK_S1A(false, false, false);
#undef NK_S1A
}

void launch_stencil32(const void* U, const Geom& g, const Stencil32Set& s, double kappa, double mu, cudaStream_t st) {
    const int nv = s.n_a + s.n_d;
    if (nv == 0) return;
    const dim3 block = s32_block(nv);
    const unsigned grid = (unsigned)((g.V + block.x - 1) / block.x);
    k_stencil32<<<grid, block, s32_smem(block.x, block.x * block.y), st>>>((const float2*)U, g, s, (float)kappa,
                                                                           (float)exp(mu), (float)exp(-mu));
}

template <bool TS, bool PASS2, bool RING>
static void launch_s1(dim3 grid, dim3 block, const float2* U, const Geom& g, const Outer& o, int j, float kappa,
                      float emu, float emu_inv, cudaStream_t st) {
    k_stencil32_step1<TS, PASS2, RING><<<grid, block, s32_smem(block.x, block.x * block.y), st>>>(U, g, o, j, kappa,
                                                                                                emu, emu_inv);
}

void launch_stencil32_step1(const void* U, const Geom& g, const Outer& o, int j, double kappa, double mu,
                            cudaStream_t st) {
    const int nv = o.two_sided ? 2 * o.n_rhs : o.n_rhs;
    const dim3 block = s32_block(nv);
    const dim3 grid((unsigned)((g.V + block.x - 1) / block.x));
    const float2* u = (const float2*)U;
    const float k = (float)kappa, ep = (float)exp(mu), em = (float)exp(-mu);
    const bool pass2 = o.y != nullptr, ring = j >= o.ring_from;
#define NK_S1(TS_, P2_, R_) launch_s1<TS_, P2_, R_>(grid, block, u, g, o, j, k, ep, em, st)
    if (o.two_sided) {
        if (pass2) { if (ring) NK_S1(true, true, true); else NK_S1(true, true, false); }
        else { if (ring) NK_S1(true, false, true); else NK_S1(true, false, false); }
    } else {
        if (pass2) { if (ring) NK_S1(false, true, true); else NK_S1(false, true, false); }
        else { if (ring) NK_S1(false, false, true); else NK_S1(false, false, false); }
    }
#undef NK_S1
}

}  // namespace nk
