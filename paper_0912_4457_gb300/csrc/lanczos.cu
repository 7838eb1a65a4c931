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
__device__ __forceinline__ void put_copy(const Outer& o, int mode, bool left, size_t at, double2 v) {
    if (mode == kCopy32) {
        float2 f = make_float2(d2f_int(v.x), d2f_int(v.y));
        (left ? o.p32 : o.q32)[at] = f;
    } else if (mode == kCopyDF && !o.qr) {
        dfc w;
        w.x = df_from_double(v.x);
        w.y = df_from_double(v.y);
        (left ? o.pdf : o.qdf)[at] = w;
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
        put_copy(o, copy_mode, false, (size_t)rhs * o.N + i, a);
        if (p) put_copy(o, copy_mode, true, (size_t)rhs * o.N + i, a);
        if (o.qr) {
            const dfc d = dfc_of(a);
            ring_q(o, rhs, 0)[i] = d;
            if (o.two_sided) ring_p(o, rhs, 0)[i] = d;
        }
    }
}

// End of step 2: the deterministic reduction of the per-thread partial
// (r^dag r, or r^dag l two-sided) and, in the last block, beta and gamma.
template <bool TS>
__device__ __forceinline__ void step2_finish(const Outer& o, int rhs, int j, double2 acc, double2* sh) {
    double2 part = block_sum(acc, sh);
    if (finish_partial(part, o.partials + (size_t)rhs * o.npart, o.counters + rhs, blockIdx.x, o.nblk)) {
        double2 d = sum_partials(o.partials + (size_t)rhs * o.npart, o.nblk, sh);
        if (threadIdx.x == 0) {
            const size_t at = (size_t)rhs * o.k + j;
            if (!TS) {
                double b = sqrt(d.x);                   // beta <- sqrt(r^dag r)
                o.beta[at] = mk(b, 0.0);
                o.gamma[at] = mk(b, 0.0);
                if (!(b > 0.0) || !isfinite(b)) o.status[rhs] = kStatusBreakdown;
            } else if ((d.x == 0.0 && d.y == 0.0) || !isfinite(d.x) || !isfinite(d.y)) {
                // serious breakdown: delta = 0 (App. B); a non-finite delta is treated alike
                o.status[rhs] = kStatusBreakdown;
                o.beta[at] = mk(0.0, 0.0);
                o.gamma[at] = mk(0.0, 0.0);
            } else {
                double2 b = csqrt_principal(d);         // beta <- sqrt(delta)
                o.beta[at] = b;
                o.gamma[at] = cdiv(cconj(d), b);        // gamma <- delta^* / beta
            }
            o.counters[rhs] = 0u;
        }
    }
}

// write_ring: also store two-float copies of the new vectors in the rings
// (read by a two-float stencil or by the two-float recurrence later on).
template <bool TS>
__global__ void __launch_bounds__(kThreads) k_step2(Outer o, int j, int copy_mode, int write_ring) {
    __shared__ double2 sh[33];
    __shared__ double2 coef[2];
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const size_t hb = (size_t)rhs * o.k;
    // H(j,j)/n_j and H(j,j)^*/m_j, one FP64 division each, by lane 0 of two
    // warps (on two SM sub-partitions) at the same time
    if ((threadIdx.x & 31) == 0 && threadIdx.x < 64) {
        const double2 a = o.alpha[hb + j];
        coef[threadIdx.x >> 5] = threadIdx.x == 0 ? cdiv(a, scale_n(o, rhs, j))
                                                  : (TS ? cdiv(cconj(a), scale_m(o, rhs, j)) : mk(0.0, 0.0));
    }
    __syncthreads();
    const double2 c3 = coef[0], c4 = coef[1];
    const double2* __restrict__ qj = outer_q(o, rhs, j);
    double2* __restrict__ r = outer_q(o, rhs, j + 1);
    const double2* __restrict__ pj = TS ? outer_p(o, rhs, j) : nullptr;
    double2* __restrict__ l = TS ? outer_p(o, rhs, j + 1) : nullptr;
    const size_t vb = (size_t)rhs * o.N;
    double2 acc = mk(0.0, 0.0);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < o.N; i += (long)o.nblk * blockDim.x) {
        const double2 q = qj[i];
        double2 rr = r[i];
        // r <- r - c3 q, l <- l - c4 p with explicit FMA
        if (TS) rr = mk(fma(-c3.x, q.x, fma(c3.y, q.y, rr.x)), fma(-c3.x, q.y, fma(-c3.y, q.x, rr.y)));
        else rr = mk(fma(-c3.x, q.x, rr.x), fma(-c3.x, q.y, rr.y));
        r[i] = rr;
        put_copy(o, copy_mode, false, vb + i, rr);
        if (write_ring) ring_q(o, rhs, j + 1)[i] = dfc_of(rr);
        if (TS) {
            const double2 pv = pj[i];
            double2 ll = l[i];
            ll = mk(fma(-c4.x, pv.x, fma(c4.y, pv.y, ll.x)), fma(-c4.x, pv.y, fma(-c4.y, pv.x, ll.y)));
            l[i] = ll;
            put_copy(o, copy_mode, true, vb + i, ll);
            if (write_ring) ring_p(o, rhs, j + 1)[i] = dfc_of(ll);
            acc.x = fma(rr.x, ll.x, fma(rr.y, ll.y, acc.x));   // conj(r) l
            acc.y = fma(rr.x, ll.y, fma(-rr.y, ll.x, acc.y));
        } else {
            acc.x = fma(rr.x, rr.x, fma(rr.y, rr.y, acc.x));
        }
    }
    step2_finish<TS>(o, rhs, j, acc, sh);
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
    __shared__ double2 coef[2];
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const size_t hb = (size_t)rhs * o.k;
    // H(j,j)/n_j and H(j,j)^*/m_j, one FP64 division each, by lane 0 of two
    // warps (on two SM sub-partitions) at the same time
    if ((threadIdx.x & 31) == 0 && threadIdx.x < 64) {
        const double2 a = o.alpha[hb + j];
        coef[threadIdx.x >> 5] = threadIdx.x == 0 ? cdiv(a, scale_n(o, rhs, j))
                                                  : (TS ? cdiv(cconj(a), scale_m(o, rhs, j)) : mk(0.0, 0.0));
    }
    __syncthreads();
    const dfc c3 = dfc_of(coef[0]), c4 = dfc_of(coef[1]);
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
            if (copy_mode == kCopy32) o.q32[vb + i] = make_float2(a.x.hi, a.y.hi);
            if (TS) {
                dfc& b = ll[u];
                b.x = b.x - (c4.x * pv[u].x - c4.y * pv[u].y);
                b.y = b.y - (c4.x * pv[u].y + c4.y * pv[u].x);
                l[i] = b;
                if (copy_mode == kCopy32) o.p32[vb + i] = make_float2(b.x.hi, b.y.hi);
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

void launch_adapt_delta(const Outer& o, const double2* c, double2* c_prev, int k, double2* dn, cudaStream_t st) {
    k_adapt_delta<<<o.n_rhs, 256, 0, st>>>(o, c, c_prev, k, dn);
}

}  // namespace nk
