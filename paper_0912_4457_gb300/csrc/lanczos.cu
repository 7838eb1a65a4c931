// Outer Krylov recurrence on the 12V-dimensional vectors, batched over RHS:
// Lanczos (App. A, mu = 0) and two-sided Lanczos (App. B, mu != 0), and the
// lift y = |x| V_k c (Eq. nested, App. C step 6).
//
// GB300 layout of the recurrence.  The basis is kept UNNORMALISED: the stored
// right vector is q_j = n_j v_j with n_0 = |x|, n_{j+1} = beta_j (so q_{j+1} is
// the residual r of step j itself), and the left vector p_j = m_j w_j with
// m_0 = |x|, m_{j+1} = gamma_j^*.  Every normalisation of App. A / B becomes a
// scalar folded into a coefficient, which removes the "v <- r / beta" pass
// and a third of the FP64 operations per vector element (FP64 is the scarce
// unit on GB300).  In exact arithmetic this is the paper's recurrence; the
// coefficients alpha, beta, gamma are the entries of H_k as App. A / B define
// them.  One outer step j is two kernels:
//   dslash_step1 (dslash.cu): s = A q_j / n_j (and t = A^dag p_j / m_j), then
//          r = s - (c_{j-1}/n_{j-1}) q_{j-1},  l = t - (beta^*_{j-1}/m_{j-1}) p_{j-1}
//          H(j,j) = v_j^dag r (= w_j^dag r two-sided), stored r -> q_{j+1}, l -> p_{j+1};
//   step2: r <- r - (H(j,j)/n_j) q_j,  l <- l - (H(j,j)^*/m_j) p_j,
//          beta = |r| (two-sided: delta = r^dag l, beta = sqrt(delta),
//          gamma = delta^*/beta; delta = 0 is a serious breakdown),
//          plus the FP32 copies the next mixed-precision stencil reads.
// In the mixed schedule, from the step where its recurrence turns two-float,
// both kernels work in two-float arithmetic on rings of the newest three
// right and left vectors (k_step2_df), and the basis columns they produce are
// stored as two-float values.
//
// Reductions are deterministic: a fixed grid, a fixed per-thread order,
// warp-shuffle and shared-memory block sums, per-block partials and a final
// fixed-order sum in the last block to finish (integer ticket, no
// floating-point atomics).  The same launch configuration therefore
// regenerates bit-identical coefficients, which the double-pass mode relies on.
#include "nk_common.cuh"
#include "nk_kernels.h"

namespace nk {

namespace {

constexpr int kThreads = 256;


__global__ void __launch_bounds__(kThreads) k_norm(Outer o, int keep_status) {
    __shared__ double2 sh[33];
    const int rhs = blockIdx.y;
    const double2* x = outer_q(o, rhs, 0);
    double acc = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < o.N; i += (long)o.nblk * blockDim.x) {
        double2 v = x[i];
        acc += v.x * v.x + v.y * v.y;
    }
    double2 part = block_sum(mk(acc, 0.0), sh);
    if (finish_partial(part, o.partials + (size_t)rhs * o.npart, o.counters + rhs, blockIdx.x, o.nblk)) {
        double2 tot = sum_partials(o.partials + (size_t)rhs * o.npart, o.nblk, sh);
        if (threadIdx.x == 0) {
            double nrm = sqrt(tot.x);
            o.xnorm[rhs] = nrm;
            // the second pass of NK_DOUBLE_PASS keeps a failure of the first
            // (breakdown, RHi): that source is not recomputed
            const int prev = o.status[rhs];
            const bool keep = keep_status && prev != kStatusOK && prev != kStatusZeroSource;
            o.status[rhs] = keep ? prev : (nrm > 0.0 ? kStatusOK : kStatusZeroSource);
            o.counters[rhs] = 0u;
            // scalars of step 0: n_0 = m_0 = |x|, no previous vector
            double2* sc = o.sc + (size_t)rhs * kScalars;
            const double2 inv = nrm > 0.0 ? cinv(mk(nrm, 0.0)) : mk(0.0, 0.0);
            sc[kScN] = inv;
            sc[kScC1] = mk(0.0, 0.0);
            sc[kScD] = inv;
            sc[kScM] = inv;
            sc[kScC1L] = mk(0.0, 0.0);
        }
    }
}

__device__ __forceinline__ dfc dfc_of(double2 v) {
    dfc r;
    r.x = df_from_double(v.x);
    r.y = df_from_double(v.y);
    return r;
}
__device__ __forceinline__ double2 double2_of(dfc v) { return mk(df_to_double(v.x), df_to_double(v.y)); }

// The next stencil's input copy of one element (FP32 or two-float), made on
// the integer pipe.  With the mixed schedule's rings the two-float copy is not
// made here (the FP64 steps write the rings themselves, which the two-float
// stencil reads).
// Element i = c V + s of RHS rhs (FP64 layout [12][V]); the FP32 copy goes to
// the pair layout.
__device__ __forceinline__ void put_copy(const Outer& o, int mode, bool left, int rhs, long i, double2 v) {
    if (mode == kCopy32) {
        const int V = (int)(o.N / 12);
        const int c = (int)(i / V), s = (int)(i - (long)c * V);
        float2 f = make_float2(d2f_int(v.x), d2f_int(v.y));
        reinterpret_cast<float2*>(left ? o.p32 : o.q32)[(size_t)rhs * o.N + f32_pair_index(c, s, V)] = f;
    } else if (mode == kCopyDF && !o.qr) {
        dfc w;
        w.x = df_from_double(v.x);
        w.y = df_from_double(v.y);
        (left ? o.pdf : o.qdf)[(size_t)rhs * o.N + i] = w;
    }
}

// q_0 = x is already in place; p_0 = x, and the copies the first stencil reads.
// Mixed schedule: the two-float rings hold q_0 and p_0, and a two-float
// stencil reads the ring itself.
__global__ void __launch_bounds__(kThreads) k_init(Outer o, int copy_mode) {
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const double2* x = outer_q(o, rhs, 0);
    double2* p = o.two_sided ? outer_p(o, rhs, 0) : nullptr;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < o.N; i += (long)o.nblk * blockDim.x) {
        double2 a = x[i];
        if (p) p[i] = a;
        put_copy(o, copy_mode, false, rhs, i, a);
        if (p) put_copy(o, copy_mode, true, rhs, i, a);
        if (o.qr) {
            const dfc d = dfc_of(a);
            ring_q(o, rhs, 0)[i] = d;
            if (o.two_sided) ring_p(o, rhs, 0)[i] = d;
        }
    }
}

// End of step 2: the deterministic reduction of the per-thread partial
// (r^dag r, or r^dag l two-sided) and, in the last block, beta and gamma and
// the scalars of step j + 1 (one complex division per warp, side by side on
// the SM sub-partitions).
template <bool TS>
__device__ __forceinline__ void step2_finish(const Outer& o, int rhs, int j, double2 acc, double2* sh) {
    __shared__ double2 bg[2];
    double2 part = block_sum(acc, sh);
    if (finish_partial(part, o.partials + (size_t)rhs * o.npart, o.counters + rhs, blockIdx.x, o.nblk)) {
        double2 d = sum_partials(o.partials + (size_t)rhs * o.npart, o.nblk, sh);
        if (threadIdx.x == 0) {
            const size_t at = (size_t)rhs * o.k + j;
            double2 b, g;
            if (!TS) {
                const double bb = sqrt(d.x);             // beta <- sqrt(r^dag r)
                b = g = mk(bb, 0.0);
                if (!(bb > 0.0) || !isfinite(bb)) o.status[rhs] = kStatusBreakdown;
            } else if ((d.x == 0.0 && d.y == 0.0) || !isfinite(d.x) || !isfinite(d.y)) {
                // serious breakdown: delta = 0 (App. B); a non-finite delta is treated alike
                o.status[rhs] = kStatusBreakdown;
                b = g = mk(0.0, 0.0);
            } else {
                b = csqrt_principal(d);                  // beta <- sqrt(delta)
                g = cdiv(cconj(d), b);                   // gamma <- delta^* / beta
            }
            o.beta[at] = b;
            o.gamma[at] = g;
            bg[0] = b;
            bg[1] = g;
            o.counters[rhs] = 0u;
        }
        __syncthreads();
        // step j + 1: n_{j+1} = beta_j, m_{j+1} = gamma_j^*
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0 && w < 5 && j + 1 < o.k && o.status[rhs] == kStatusOK) {
            const double2 b = bg[0], g = bg[1];
            double2* sc = o.sc + (size_t)rhs * kScalars;
            if (w == 0) sc[kScN] = cinv(b);
            else if (w == 1) sc[kScC1] = cdiv(TS ? g : b, scale_n(o, rhs, j));
            else if (w == 2) sc[kScD] = TS ? cinv(g) : cinv(b);
            else if (w == 3) sc[kScM] = cinv(cconj(g));
            else sc[kScC1L] = cdiv(cconj(b), scale_m(o, rhs, j));
        }
    }
}

// FP64 step 2 (the recurrence of NK_FP64 and of the mixed schedule):
//   r <- r - (H(j,j)/n_j) q_j,  l <- l - (H(j,j)^*/m_j) p_j,  delta += r^dag l,
// plus the copies the next stencil reads (FP32 pair layout; write_ring: also
// two-float copies in the rings for a two-float stencil or a later ring
// step).  Each thread takes a spin-colour component pair (2i, 2i + 1) of a
// site -- the elements i V + s ... of the FP64 layout and one float4 of the
// FP32 copy -- two pairs per iteration with every load issued first (the
// kernel is bound by the FP64 pipe and by the latency of these loads).
template <bool TS>
__global__ void __launch_bounds__(kThreads) k_step2(Outer o, int j, int copy_mode, int write_ring) {
    __shared__ double2 sh[33];
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const double2 c3 = o.sc[(size_t)rhs * kScalars + kScC3];
    const double2 c4 = o.sc[(size_t)rhs * kScalars + kScC4];
    const unsigned V = (unsigned)(o.N / 12);
    const unsigned NP = 6u * V;
    const double2* __restrict__ qj = outer_q(o, rhs, j);
    double2* __restrict__ r = outer_q(o, rhs, j + 1);
    const double2* __restrict__ pj = TS ? outer_p(o, rhs, j) : nullptr;
    double2* __restrict__ l = TS ? outer_p(o, rhs, j + 1) : nullptr;
    float4* __restrict__ r32 = o.q32 + (size_t)rhs * NP;
    float4* __restrict__ l32 = TS ? o.p32 + (size_t)rhs * NP : nullptr;
    dfc* __restrict__ rr_ring = write_ring ? ring_q(o, rhs, j + 1) : nullptr;
    dfc* __restrict__ ll_ring = (write_ring && TS) ? ring_p(o, rhs, j + 1) : nullptr;
    constexpr int U = 2;
    const unsigned stride = (unsigned)o.nblk * blockDim.x;
    double2 acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = mk(0.0, 0.0);
    for (unsigned p0 = blockIdx.x * blockDim.x + threadIdx.x; p0 < NP; p0 += U * stride) {
        double2 q[U][2], rv[U][2], pv[U][2], lv[U][2];
        size_t e[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned p = p0 + u * stride;
            const unsigned cp = p / V, s = p - cp * V;
            e[u] = (size_t)(2 * cp) * V + s;
            if (p < NP) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    q[u][h] = qj[e[u] + h * V];
                    rv[u][h] = r[e[u] + h * V];
                    if (TS) { pv[u][h] = pj[e[u] + h * V]; lv[u][h] = l[e[u] + h * V]; }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned p = p0 + u * stride;
            if (p >= NP) break;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                double2 a = rv[u][h];
                const double2 qq = q[u][h];
                // r <- r - c3 q, l <- l - c4 p with explicit FMA
                if (TS) a = mk(fma(-c3.x, qq.x, fma(c3.y, qq.y, a.x)), fma(-c3.x, qq.y, fma(-c3.y, qq.x, a.y)));
                else a = mk(fma(-c3.x, qq.x, a.x), fma(-c3.x, qq.y, a.y));
                rv[u][h] = a;
                r[e[u] + h * V] = a;
                if (rr_ring) rr_ring[e[u] + h * V] = dfc_of(a);
                if (TS) {
                    double2 b = lv[u][h];
                    const double2 pp = pv[u][h];
                    b = mk(fma(-c4.x, pp.x, fma(c4.y, pp.y, b.x)), fma(-c4.x, pp.y, fma(-c4.y, pp.x, b.y)));
                    lv[u][h] = b;
                    l[e[u] + h * V] = b;
                    if (ll_ring) ll_ring[e[u] + h * V] = dfc_of(b);
                    acc[u].x = fma(a.x, b.x, fma(a.y, b.y, acc[u].x));   // conj(r) l
                    acc[u].y = fma(a.x, b.y, fma(-a.y, b.x, acc[u].y));
                } else {
                    acc[u].x = fma(a.x, a.x, fma(a.y, a.y, acc[u].x));
                }
            }
            if (copy_mode == kCopy32) {
                r32[p] = make_float4(d2f_int(rv[u][0].x), d2f_int(rv[u][0].y), d2f_int(rv[u][1].x),
                                     d2f_int(rv[u][1].y));
                if (TS) l32[p] = make_float4(d2f_int(lv[u][0].x), d2f_int(lv[u][0].y), d2f_int(lv[u][1].x),
                                             d2f_int(lv[u][1].y));
            }
        }
    }
    double2 tot = acc[0];
#pragma unroll
    for (int u = 1; u < U; ++u) { tot.x += acc[u].x; tot.y += acc[u].y; }
    step2_finish<TS>(o, rhs, j, tot, sh);
}

// Step 2 of the late (FP32-stencil) steps of the mixed schedule in two-float
// arithmetic on the FP32 pipe, on the two-float rings: r and l (left in ring slot j + 1
// by the stencil kernel) are updated with q_j and p_j from the rings; r is
// also written to the basis Q (as two-float values in a single-pass solve,
// else FP64: one FP64 addition per component), and the
// FP32 copy the next FP32 stencil reads is the high part (a two-float
// stencil reads the ring).  The FP32 stencil of the late steps perturbs the
// recurrence at 1e-7; 48-bit arithmetic adds about 1e-14.  The all-FP64
// schedule (NK_FP64) keeps k_step2.
template <bool TS>
__global__ void __launch_bounds__(kThreads, 2) k_step2_df(Outer o, int j, int copy_mode) {
    __shared__ double2 sh[33];
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const dfc c3 = dfc_of(o.sc[(size_t)rhs * kScalars + kScC3]);
    const dfc c4 = dfc_of(o.sc[(size_t)rhs * kScalars + kScC4]);
    const int V = (int)(o.N / 12);
    const dfc* __restrict__ qj = ring_q(o, rhs, j);
    dfc* __restrict__ r = ring_q(o, rhs, j + 1);
    double2* __restrict__ rq = outer_q(o, rhs, j + 1);
    const bool qdf = j + 1 >= o.q_df_from;   // the basis column is kept in two-float form
    const dfc* __restrict__ pj = TS ? ring_p(o, rhs, j) : nullptr;
    dfc* __restrict__ l = TS ? ring_p(o, rhs, j + 1) : nullptr;
    const size_t vb = (size_t)rhs * o.N;
    // U elements per thread and iteration, all their loads issued before any
    // arithmetic (the kernel is bound by the latency of these L2 reads), one
    // accumulator each
    constexpr int U = 4;
    df ax[U], ay[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ax[u] = ay[u] = df(0);
    const long stride = (long)o.nblk * blockDim.x;
    for (long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x; i0 < o.N; i0 += U * stride) {
        dfc q[U], rr[U], pv[U], ll[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long i = i0 + u * stride;
            if (i < o.N) {
                q[u] = qj[i];
                rr[u] = r[i];
                if (TS) { pv[u] = pj[i]; ll[u] = l[i]; }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long i = i0 + u * stride;
            if (i >= o.N) break;
            // r <- r - c3 q, l <- l - c4 p
            dfc& a = rr[u];
            if (TS) {
                a.x = a.x - (c3.x * q[u].x - c3.y * q[u].y);
                a.y = a.y - (c3.x * q[u].y + c3.y * q[u].x);
            } else {
                a.x = a.x - c3.x * q[u].x;
                a.y = a.y - c3.x * q[u].y;
            }
            r[i] = a;
            if (qdf) reinterpret_cast<dfc*>(rq)[i] = a;
            else rq[i] = double2_of(a);
            const int c = (int)(i / V), site = (int)(i - (long)c * V);
            const size_t i32 = vb + f32_pair_index(c, site, V);
            if (copy_mode == kCopy32) reinterpret_cast<float2*>(o.q32)[i32] = make_float2(a.x.hi, a.y.hi);
            if (TS) {
                dfc& b = ll[u];
                b.x = b.x - (c4.x * pv[u].x - c4.y * pv[u].y);
                b.y = b.y - (c4.x * pv[u].y + c4.y * pv[u].x);
                l[i] = b;
                if (copy_mode == kCopy32) reinterpret_cast<float2*>(o.p32)[i32] = make_float2(b.x.hi, b.y.hi);
                ax[u] += a.x * b.x + a.y * b.y;   // conj(r) l
                ay[u] += a.x * b.y - a.y * b.x;
            } else {
                ax[u] += a.x * a.x + a.y * a.y;
            }
        }
    }
    step2_finish<TS>(o, rhs, j, mk(df_to_double((ax[0] + ax[1]) + (ax[2] + ax[3])),
                                   df_to_double((ay[0] + ay[1]) + (ay[2] + ay[3]))), sh);
}

// c'_j = |x| c_j / n_j: the lift coefficients on the unnormalised basis
// (zero from kused on, where the basis and its scales were never computed).
__global__ void k_lift_coef(Outer o, const double2* __restrict__ c, const int* __restrict__ kused,
                            double2* __restrict__ cp) {
    const int rhs = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= o.k) return;
    double2* out = cp + (size_t)rhs * o.k;
    if (o.status[rhs] != kStatusOK || j >= kused[rhs]) { out[j] = mk(0.0, 0.0); return; }
    out[j] = cscale(cdiv(c[(size_t)rhs * o.k + j], scale_n(o, rhs, j)), o.xnorm[rhs]);
}

// per RHS: dn = (|c - c_prev|, |c|) over the first k entries; then c_prev <- c
__global__ void k_adapt_delta(Outer o, const double2* __restrict__ c, double2* __restrict__ cprev, int k,
                              double2* __restrict__ dn) {
    __shared__ double2 sh[33];
    const int rhs = blockIdx.x;
    if (o.status[rhs] != kStatusOK) return;   // frozen or failed: keep its accepted c
    const double2* cr = c + (size_t)rhs * o.k;
    double2* pr = cprev + (size_t)rhs * o.k;
    double d = 0.0, n = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double2 a = cr[j], b = pr[j];
        d += cnorm2(csub(a, b));
        n += cnorm2(a);
    }
    double2 t = block_sum(mk(d, n), sh);
    for (int j = threadIdx.x; j < k; j += blockDim.x) pr[j] = cr[j];
    if (threadIdx.x == 0) dn[rhs] = mk(sqrt(t.x), sqrt(t.y));
}

// y_r = sum_j c'_r[j] q_j  (reads every basis vector once)
__global__ void __launch_bounds__(kThreads) k_lift(Outer o, const double2* __restrict__ cp,
                                                    const int* __restrict__ kused, double2* __restrict__ y) {
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= o.N) return;
    double2* yo = y + (size_t)rhs * o.N;
    if (o.status[rhs] != kStatusOK) { yo[i] = mk(0.0, 0.0); return; }
    const double2* cr = cp + (size_t)rhs * o.k;
    const double2* Qr = o.Q + (size_t)rhs * o.qcols * o.N;
    const int ku = kused[rhs];
    double2 acc = mk(0.0, 0.0);
    for (int j = 0; j < ku; ++j) {
        double2 cj = __ldg(cr + j);
        double2 v = Qr[(size_t)j * o.N + i];
        acc.x += cj.x * v.x - cj.y * v.y;
        acc.y += cj.x * v.y + cj.y * v.x;
    }
    yo[i] = acc;
}

// The same lift in two-float arithmetic for the mixed schedule: the
// coefficients are converted once per block into shared memory, each basis
// element on load, and the sum runs in two accumulators (even and odd j).
__global__ void __launch_bounds__(kThreads) k_lift_df(Outer o, const double2* __restrict__ cp,
                                                       const int* __restrict__ kused, double2* __restrict__ y) {
    extern __shared__ dfc cs[];   // [kused]
    const int rhs = blockIdx.y;
    const int ku = kused[rhs];
    const double2* cr = cp + (size_t)rhs * o.k;
    for (int j = threadIdx.x; j < ku; j += blockDim.x) cs[j] = dfc_of(cr[j]);
    __syncthreads();
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= o.N) return;
    double2* yo = y + (size_t)rhs * o.N;
    if (o.status[rhs] != kStatusOK) { yo[i] = mk(0.0, 0.0); return; }
    const double2* Qr = o.Q + (size_t)rhs * o.qcols * o.N;
    dfc acc[2];
    acc[0].x = df(0); acc[0].y = df(0); acc[1] = acc[0];
    const int j1 = min(ku, o.q_df_from);   // columns [j1, ku) are two-float already
    for (int j = 0; j < ku; ++j) {
        const dfc c = cs[j];
        const dfc v = j < j1 ? dfc_of(Qr[(size_t)j * o.N + i]) : reinterpret_cast<const dfc*>(Qr)[(size_t)j * o.N + i];
        dfc& a = acc[j & 1];
        a.x += c.x * v.x - c.y * v.y;
        a.y += c.x * v.y + c.y * v.x;
    }
    dfc t;
    t.x = acc[0].x + acc[1].x;
    t.y = acc[0].y + acc[1].y;
    yo[i] = double2_of(t);
}

// double pass: zero the status of sources that are exactly zero
__global__ void k_zero_bad(Outer o, double2* y) {
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= o.N) return;
    if (o.status[rhs] != kStatusOK) y[(size_t)rhs * o.N + i] = mk(0.0, 0.0);
}

}  // namespace

void launch_outer_init(const Outer& o, int copy_mode, cudaStream_t st, bool keep_status) {
    dim3 grid(o.nblk, o.n_rhs);
    k_norm<<<grid, kThreads, 0, st>>>(o, keep_status ? 1 : 0);
    k_init<<<grid, kThreads, 0, st>>>(o, copy_mode);
}

void launch_outer_step2(const Outer& o, int j, int copy_mode, bool ring, bool write_ring, cudaStream_t st) {
    dim3 grid(o.nblk, o.n_rhs);
    const int wr = (write_ring && o.qr) ? 1 : 0;
    if (!ring || !o.qr) {   // FP64 step
        if (o.two_sided) k_step2<true><<<grid, kThreads, 0, st>>>(o, j, copy_mode, wr);
        else k_step2<false><<<grid, kThreads, 0, st>>>(o, j, copy_mode, wr);
    } else {
        if (o.two_sided) k_step2_df<true><<<grid, kThreads, 0, st>>>(o, j, copy_mode);
        else k_step2_df<false><<<grid, kThreads, 0, st>>>(o, j, copy_mode);
    }
}

void launch_lift_coef(const Outer& o, const double2* c, const int* kused, double2* cp, cudaStream_t st) {
    dim3 grid((o.k + 127) / 128, o.n_rhs);
    k_lift_coef<<<grid, 128, 0, st>>>(o, c, kused, cp);
}

void launch_lift(const Outer& o, const double2* cp, const int* kused, double2* y, cudaStream_t st) {
    dim3 grid((unsigned)((o.N + kThreads - 1) / kThreads), o.n_rhs);
    // the two-float lift only where the two-float recurrence wrote two-float
    // basis columns; an FP64 recurrence is lifted in FP64
    if (o.q_ring) k_zero_bad<<<grid, kThreads, 0, st>>>(o, y);
    else if (o.qr && o.q_df_from < o.k) k_lift_df<<<grid, kThreads, sizeof(dfc) * (size_t)o.k, st>>>(o, cp, kused, y);
    else k_lift<<<grid, kThreads, 0, st>>>(o, cp, kused, y);
}

__global__ void k_fill_int(int* p, int n, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

void launch_fill_int(int* p, int n, int value, cudaStream_t st) {
    k_fill_int<<<(n + 127) / 128, 128, 0, st>>>(p, n, value);
}

// per RHS r: (|x2_r - b_r|^2, |b_r|^2), one block per RHS, fixed-order sums
__global__ void k_eps_sums(const double2* __restrict__ b, const double2* __restrict__ x2, long N,
                           double2* __restrict__ out) {
    __shared__ double2 sh[33];
    const size_t base = (size_t)blockIdx.x * N;
    double d = 0.0, n = 0.0;
    for (long i = threadIdx.x; i < N; i += blockDim.x) {
        const double2 a = b[base + i], c = x2[base + i];
        d += cnorm2(csub(c, a));
        n += cnorm2(a);
    }
    const double2 t = block_sum(mk(d, n), sh);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
}

void launch_eps_sums(const double2* b, const double2* x2, int n, long N, double2* out, cudaStream_t st) {
    k_eps_sums<<<n, 1024, 0, st>>>(b, x2, N, out);
}

void launch_adapt_delta(const Outer& o, const double2* c, double2* c_prev, int k, double2* dn, cudaStream_t st) {
    k_adapt_delta<<<o.n_rhs, 256, 0, st>>>(o, c, c_prev, k, dn);
}

}  // namespace nk
