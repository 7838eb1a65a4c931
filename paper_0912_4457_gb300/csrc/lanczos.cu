// Outer Krylov recurrence on the 12V-dimensional vectors, batched over RHS:
// Lanczos (App. A, mu = 0) and two-sided Lanczos (App. B, mu != 0), plus the
// lift y = |x| V_k c (Eq. nested, App. C step 6).
//
// One outer step j is split at its two global reductions:
//   step1: r <- A v_j - c_{j-1} v_{j-1}      (c = beta, two-sided: gamma)
//          l <- A^dag w_j - beta*_{j-1} w_{j-1}           (two-sided only)
//          H(j,j) <- v_j^dag r  (two-sided: w_j^dag r)
//   step2: r <- r - H(j,j) v_j,  l <- l - H(j,j)^* w_j
//          beta <- sqrt(r^dag r)  (two-sided: delta = r^dag l, beta = sqrt(delta),
//          gamma = delta^* / beta; delta = 0 is a serious breakdown)
//   step3: v_{j+1} <- r / beta,  w_{j+1} <- l / gamma^*
// The stencil output A v_j (and A^dag w_j) comes from dslash.cu.
//
// Reductions are deterministic: a fixed grid (nblk blocks per RHS) with a
// fixed per-thread order, warp-shuffle and shared-memory block sums, per-block
// partials, and a final fixed-order sum in the last block to finish (found
// with an integer atomic ticket; no floating-point atomics).  The same
// launch configuration therefore regenerates bit-identical coefficients,
// which the double-pass mode relies on.
#include "nk_common.cuh"
#include "nk_kernels.h"

namespace nk {

namespace {

constexpr int kThreads = 256;

// Writes this block's partial, and returns true in the block that finishes last.
__device__ __forceinline__ bool finish_partial(double2 part, double2* partials, unsigned* counter,
                                               int nblk) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = part;
        __threadfence();
        unsigned ticket = atomicAdd(counter, 1u);
        last = (ticket == (unsigned)nblk - 1u);
    }
    __syncthreads();
    return last;
}

// Fixed-order sum of the nblk partials (called by all threads of the last block).
__device__ __forceinline__ double2 sum_partials(const double2* partials, int nblk, double2* sh) {
    __threadfence();
    double2 a = mk(0.0, 0.0);
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        double2 v = __ldcg(partials + i);
        a.x += v.x; a.y += v.y;
    }
    return block_sum(a, sh);
}

__global__ void __launch_bounds__(kThreads) k_norm(Outer o, const double2* __restrict__ b) {
    __shared__ double2 sh[32];
    const int rhs = blockIdx.y;
    const double2* x = b + (size_t)rhs * o.N;
    double acc = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < o.N; i += (long)o.nblk * blockDim.x) {
        double2 v = x[i];
        acc += v.x * v.x + v.y * v.y;
    }
    double2 part = block_sum(mk(acc, 0.0), sh);
    if (finish_partial(part, o.partials + (size_t)rhs * o.nblk, o.counters + rhs, o.nblk)) {
        double2 tot = sum_partials(o.partials + (size_t)rhs * o.nblk, o.nblk, sh);
        if (threadIdx.x == 0) {
            double nrm = sqrt(tot.x);
            o.xnorm[rhs] = nrm;
            o.status[rhs] = nrm > 0.0 ? kStatusOK : kStatusZeroSource;
            o.counters[rhs] = 0u;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_init(Outer o, const double2* __restrict__ b, int write32) {
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const double inv = 1.0 / o.xnorm[rhs];
    const double2* x = b + (size_t)rhs * o.N;
    double2* v = outer_v(o, rhs, 0);
    double2* w = o.two_sided ? outer_w(o, rhs, 0) : nullptr;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < o.N; i += (long)o.nblk * blockDim.x) {
        double2 a = x[i];
        double2 vv = mk(a.x * inv, a.y * inv);   // v_1 <- x / |x|
        v[i] = vv;
        if (w) w[i] = vv;                        // w_1 <- v_1
        if (write32) {
            float2 f = make_float2((float)vv.x, (float)vv.y);
            o.v32[(size_t)rhs * o.N + i] = f;
            if (w) o.w32[(size_t)rhs * o.N + i] = f;
        }
    }
}

template <bool TS>
__global__ void __launch_bounds__(kThreads) k_step1(Outer o, int j) {
    __shared__ double2 sh[32];
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const size_t base = (size_t)rhs * o.N;
    const double2* __restrict__ vj = outer_v(o, rhs, j);
    const double2* __restrict__ vjm = j > 0 ? outer_v(o, rhs, j - 1) : nullptr;
    const double2* __restrict__ wj = TS ? outer_w(o, rhs, j) : nullptr;
    const double2* __restrict__ wjm = (TS && j > 0) ? outer_w(o, rhs, j - 1) : nullptr;
    const double2* __restrict__ s = o.s + base;
    const double2* __restrict__ t = TS ? o.t + base : nullptr;
    double2* __restrict__ r = o.r + base;
    double2* __restrict__ l = TS ? o.l + base : nullptr;
    double2 cprev = mk(0.0, 0.0), bprevc = mk(0.0, 0.0);
    if (j > 0) {
        cprev = TS ? o.gamma[(size_t)rhs * o.k + j - 1] : o.beta[(size_t)rhs * o.k + j - 1];
        bprevc = cconj(o.beta[(size_t)rhs * o.k + j - 1]);
    }
    // double-pass accumulation y += c_j v_j
    double2* __restrict__ y = o.y ? o.y + base : nullptr;
    const double2 cj = o.y ? o.c[(size_t)rhs * o.k + j] : mk(0.0, 0.0);
    double2 acc = mk(0.0, 0.0);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < o.N; i += (long)o.nblk * blockDim.x) {
        double2 rr = s[i];
        if (j > 0) {
            double2 vp = vjm[i];
            if (TS) rr = csub(rr, cmul(cprev, vp));
            else rr = mk(rr.x - cprev.x * vp.x, rr.y - cprev.x * vp.y);
        }
        r[i] = rr;
        if (TS) {
            double2 ll = t[i];
            if (j > 0) ll = csub(ll, cmul(bprevc, wjm[i]));
            l[i] = ll;
            double2 ww = wj[i];
            acc.x += ww.x * rr.x + ww.y * rr.y;   // conj(w) r
            acc.y += ww.x * rr.y - ww.y * rr.x;
        } else {
            double2 vv = vj[i];
            acc.x += vv.x * rr.x + vv.y * rr.y;   // Re(conj(v) r)
        }
        if (y) y[i] = cadd(y[i], cmul(cj, vj[i]));
    }
    double2 part = block_sum(acc, sh);
    if (finish_partial(part, o.partials + (size_t)rhs * o.nblk, o.counters + rhs, o.nblk)) {
        double2 tot = sum_partials(o.partials + (size_t)rhs * o.nblk, o.nblk, sh);
        if (threadIdx.x == 0) {
            if (!TS) tot.y = 0.0;  // Hermitian: H(j,j) real (App. C, "real arithmetic")
            o.alpha[(size_t)rhs * o.k + j] = tot;
            o.counters[rhs] = 0u;
        }
    }
}

template <bool TS>
__global__ void __launch_bounds__(kThreads) k_step2(Outer o, int j) {
    __shared__ double2 sh[32];
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const size_t base = (size_t)rhs * o.N;
    const double2* __restrict__ vj = outer_v(o, rhs, j);
    const double2* __restrict__ wj = TS ? outer_w(o, rhs, j) : nullptr;
    double2* __restrict__ r = o.r + base;
    double2* __restrict__ l = TS ? o.l + base : nullptr;
    const double2 a = o.alpha[(size_t)rhs * o.k + j];
    const double2 ac = cconj(a);
    double2 acc = mk(0.0, 0.0);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < o.N; i += (long)o.nblk * blockDim.x) {
        double2 v = vj[i];
        double2 rr;
        if (TS) rr = csub(r[i], cmul(a, v));
        else { double2 r0 = r[i]; rr = mk(r0.x - a.x * v.x, r0.y - a.x * v.y); }
        r[i] = rr;
        if (TS) {
            double2 ll = csub(l[i], cmul(ac, wj[i]));
            l[i] = ll;
            acc.x += rr.x * ll.x + rr.y * ll.y;   // conj(r) l
            acc.y += rr.x * ll.y - rr.y * ll.x;
        } else {
            acc.x += rr.x * rr.x + rr.y * rr.y;
        }
    }
    double2 part = block_sum(acc, sh);
    if (finish_partial(part, o.partials + (size_t)rhs * o.nblk, o.counters + rhs, o.nblk)) {
        double2 d = sum_partials(o.partials + (size_t)rhs * o.nblk, o.nblk, sh);
        if (threadIdx.x == 0) {
            const size_t at = (size_t)rhs * o.k + j;
            if (!TS) {
                double b = sqrt(d.x);
                o.beta[at] = mk(b, 0.0);
                o.gamma[at] = mk(b, 0.0);
                if (!(b > 0.0) || !isfinite(b)) o.status[rhs] = kStatusBreakdown;
            } else {
                // serious breakdown: delta = 0 (App. B); a non-finite delta is treated alike
                if ((d.x == 0.0 && d.y == 0.0) || !isfinite(d.x) || !isfinite(d.y)) {
                    o.status[rhs] = kStatusBreakdown;
                    o.beta[at] = mk(0.0, 0.0);
                    o.gamma[at] = mk(0.0, 0.0);
                } else {
                    double2 b = csqrt_principal(d);     // beta <- sqrt(delta)
                    o.beta[at] = b;
                    o.gamma[at] = cdiv(cconj(d), b);    // gamma <- delta^* / beta
                }
            }
            o.counters[rhs] = 0u;
        }
    }
}

template <bool TS>
__global__ void __launch_bounds__(kThreads) k_step3(Outer o, int j, int write32) {
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const size_t base = (size_t)rhs * o.N;
    const double2* __restrict__ r = o.r + base;
    const double2* __restrict__ l = TS ? o.l + base : nullptr;
    double2* __restrict__ vn = outer_v(o, rhs, j + 1);
    double2* __restrict__ wn = TS ? outer_w(o, rhs, j + 1) : nullptr;
    const size_t at = (size_t)rhs * o.k + j;
    const double2 binv = TS ? cinv(o.beta[at]) : mk(1.0 / o.beta[at].x, 0.0);
    const double2 ginv = TS ? cinv(cconj(o.gamma[at])) : mk(0.0, 0.0);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < o.N; i += (long)o.nblk * blockDim.x) {
        double2 rr = r[i];
        double2 v = TS ? cmul(rr, binv) : mk(rr.x * binv.x, rr.y * binv.x);   // v <- r / beta
        vn[i] = v;
        if (write32) o.v32[base + i] = make_float2((float)v.x, (float)v.y);
        if (TS) {
            double2 w = cmul(l[i], ginv);                                     // w <- l / gamma^*
            wn[i] = w;
            if (write32) o.w32[base + i] = make_float2((float)w.x, (float)w.y);
        }
    }
}

// y_r = |x_r| * sum_j c_r[j] v_j  (reads every basis vector once)
__global__ void __launch_bounds__(kThreads) k_lift(Outer o, const double2* __restrict__ c, double2* __restrict__ y) {
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= o.N) return;
    double2* yo = y + (size_t)rhs * o.N;
    if (o.status[rhs] != kStatusOK) { yo[i] = mk(0.0, 0.0); return; }
    const double2* cr = c + (size_t)rhs * o.k;
    const double2* Vr = o.V + (size_t)rhs * o.k * o.N;
    double2 acc = mk(0.0, 0.0);
    for (int j = 0; j < o.k; ++j) {
        double2 cj = __ldg(cr + j);
        double2 v = Vr[(size_t)j * o.N + i];
        acc.x += cj.x * v.x - cj.y * v.y;
        acc.y += cj.x * v.y + cj.y * v.x;
    }
    const double xn = o.xnorm[rhs];
    yo[i] = mk(acc.x * xn, acc.y * xn);
}

// double pass: y <- |x| y
__global__ void k_scale_y(Outer o) {
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= o.N) return;
    double2* yo = o.y + (size_t)rhs * o.N;
    if (o.status[rhs] != kStatusOK) { yo[i] = mk(0.0, 0.0); return; }
    const double xn = o.xnorm[rhs];
    double2 v = yo[i];
    yo[i] = mk(v.x * xn, v.y * xn);
}

}  // namespace

void launch_outer_init(const Outer& o, const double2* b_soa, int write32, cudaStream_t st) {
    dim3 grid(o.nblk, o.n_rhs);
    k_norm<<<grid, kThreads, 0, st>>>(o, b_soa);
    k_init<<<grid, kThreads, 0, st>>>(o, b_soa, write32);
}

void launch_outer_step1(const Outer& o, int j, cudaStream_t st) {
    dim3 grid(o.nblk, o.n_rhs);
    if (o.two_sided) k_step1<true><<<grid, kThreads, 0, st>>>(o, j);
    else k_step1<false><<<grid, kThreads, 0, st>>>(o, j);
}

void launch_outer_step2(const Outer& o, int j, cudaStream_t st) {
    dim3 grid(o.nblk, o.n_rhs);
    if (o.two_sided) k_step2<true><<<grid, kThreads, 0, st>>>(o, j);
    else k_step2<false><<<grid, kThreads, 0, st>>>(o, j);
}

void launch_outer_step3(const Outer& o, int j, int write32, cudaStream_t st) {
    dim3 grid(o.nblk, o.n_rhs);
    if (o.two_sided) k_step3<true><<<grid, kThreads, 0, st>>>(o, j, write32);
    else k_step3<false><<<grid, kThreads, 0, st>>>(o, j, write32);
}

void launch_lift(const Outer& o, const double2* c, double2* y, cudaStream_t st) {
    dim3 grid((unsigned)((o.N + kThreads - 1) / kThreads), o.n_rhs);
    if (o.V) {
        k_lift<<<grid, kThreads, 0, st>>>(o, c, y);
    } else {
        k_scale_y<<<grid, kThreads, 0, st>>>(o);
    }
}

}  // namespace nk
