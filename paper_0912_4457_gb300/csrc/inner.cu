// Inner half of the nested method, per RHS (App. C steps 3-5, Eqs. popt,
// precond, innersign, Roberts):
//   p      = (z_min z_max)^{-1/2}, z_max by power iteration with H_k and z_min
//            by inverse iteration with the LU of H_k (30 steps each, from the
//            normalised all-ones vector), unless p is given;
//   LU of p H_k in LAPACK gttrf form (partial pivoting; U with two super-diagonals);
//   inner (two-sided) Lanczos of size l with H_k' = [p H_k + (p H_k)^{-1}]/2 and
//            e_1, applying (p H_k)^{-1} by the gttrs back substitution and
//            p H_k by a band product (App. C step 4 (a), (b));
//   Roberts-Higham iteration S <- (S + S^{-1})/2 on the dense H_l;
//   c = V_l sgn(H_l) e_1.
// In the Hermitian case (mu = 0) all of it is real arithmetic (App. C).
//
// The inner Lanczos runs one CTA per RHS: the band products, inner products
// and axpys are spread over the CTA, the two O(k) substitution sweeps of each
// solve are a sequential chain in one thread (two threads in the two-sided
// case: H_k' v and H_k'^dagger w are independent).
//
// RHi runs one thread-block cluster per RHS: the rows of the l x l matrix
// being inverted (in-place Gauss-Jordan with partial pivoting and row
// interchanges) are spread cyclically over the cluster's CTAs and held in
// their shared memory; the pivot search, the pivot row broadcast and the row
// interchange go through distributed shared memory between two cluster
// barriers per pivot.
#include <cooperative_groups.h>

#include "nk_common.cuh"
#include "nk_kernels.h"

namespace cg = cooperative_groups;

namespace nk {

namespace {

// ---- arithmetic on T = double (real, Hermitian case) or double2 (complex) ----
__device__ __forceinline__ double t_zero(double) { return 0.0; }
__device__ __forceinline__ double2 t_zero(double2) { return mk(0.0, 0.0); }
__device__ __forceinline__ double t_from(double2 a, double) { return a.x; }
__device__ __forceinline__ double2 t_from(double2 a, double2) { return a; }
__device__ __forceinline__ double2 t_to2(double a) { return mk(a, 0.0); }
__device__ __forceinline__ double2 t_to2(double2 a) { return a; }
__device__ __forceinline__ double t_conj(double a) { return a; }
__device__ __forceinline__ double2 t_conj(double2 a) { return cconj(a); }
__device__ __forceinline__ double t_mul(double a, double b) { return a * b; }
__device__ __forceinline__ double2 t_mul(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ double t_add(double a, double b) { return a + b; }
__device__ __forceinline__ double2 t_add(double2 a, double2 b) { return cadd(a, b); }
__device__ __forceinline__ double t_sub(double a, double b) { return a - b; }
__device__ __forceinline__ double2 t_sub(double2 a, double2 b) { return csub(a, b); }
__device__ __forceinline__ double t_scale(double a, double s) { return a * s; }
__device__ __forceinline__ double2 t_scale(double2 a, double s) { return cscale(a, s); }
__device__ __forceinline__ double t_neg(double a) { return -a; }
__device__ __forceinline__ double2 t_neg(double2 a) { return mk(-a.x, -a.y); }
__device__ __forceinline__ double t_inv(double a) { return 1.0 / a; }
__device__ __forceinline__ double2 t_inv(double2 a) { return cinv(a); }
__device__ __forceinline__ double t_abs1(double a) { return fabs(a); }
__device__ __forceinline__ double t_abs1(double2 a) { return cabs1(a); }  // LAPACK CABS1
__device__ __forceinline__ double t_norm2(double a) { return a * a; }
__device__ __forceinline__ double t_norm2(double2 a) { return cnorm2(a); }
__device__ __forceinline__ bool t_iszero(double a) { return a == 0.0; }
__device__ __forceinline__ bool t_iszero(double2 a) { return a.x == 0.0 && a.y == 0.0; }
// conj(a) * b
__device__ __forceinline__ double2 t_dotc(double a, double b) { return mk(a * b, 0.0); }
__device__ __forceinline__ double2 t_dotc(double2 a, double2 b) { return cmulc(a, b); }

// Tridiagonal LU with partial pivoting, LAPACK gttrf semantics (row i and
// i+1 are interchanged when |d_i| < |dl_i|, |.| = |re| + |im| for complex).
// On return dl holds the multipliers, d, du, du2 the rows of U, ipiv the
// interchanges (0-based: ipiv[i] = i or i+1) and dinv = 1/d.
// Returns 0, or i+1 if U(i,i) = 0.  Sequential, one thread.
template <typename T>
__device__ int gttrf(int n, T* dl, T* d, T* du, T* du2, int* ipiv, T* dinv) {
    for (int i = 0; i < n; ++i) ipiv[i] = i;
    for (int i = 0; i < n - 2; ++i) du2[i] = t_zero(T());
    for (int i = 0; i < n - 1; ++i) {
        if (t_abs1(d[i]) >= t_abs1(dl[i])) {
            if (!t_iszero(d[i])) {
                T fact = t_mul(dl[i], t_inv(d[i]));
                dl[i] = fact;
                d[i + 1] = t_sub(d[i + 1], t_mul(fact, du[i]));
            }
        } else {
            T fact = t_mul(d[i], t_inv(dl[i]));
            d[i] = dl[i];
            dl[i] = fact;
            T temp = du[i];
            du[i] = d[i + 1];
            d[i + 1] = t_sub(temp, t_mul(fact, d[i + 1]));
            if (i < n - 2) {
                du2[i] = du[i + 1];
                du[i + 1] = t_mul(t_scale(fact, -1.0), du[i + 1]);
            }
            ipiv[i] = i + 1;
        }
    }
    int info = 0;
    for (int i = 0; i < n; ++i) {
        if (t_iszero(d[i])) { if (!info) info = i + 1; dinv[i] = t_zero(T()); }
        else dinv[i] = t_inv(d[i]);
    }
    return info;
}

// y = p * H x (dagger: p * H^dagger x) for the outer tridiagonal, in the
// summation order (diag, sub, super) -- all threads of the block.
template <typename T>
__device__ void band_mv(int n, double p, const double2* al, const double2* be, const double2* ga,
                        const T* __restrict__ x, T* __restrict__ y, bool dagger) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        T dg = t_from(al[i], T());
        if (dagger) dg = t_conj(dg);
        T acc = t_mul(dg, x[i]);
        if (i > 0) {
            T sub = dagger ? t_conj(t_from(ga[i - 1], T())) : t_from(be[i - 1], T());
            acc = t_add(acc, t_mul(sub, x[i - 1]));
        }
        if (i < n - 1) {
            T sup = dagger ? t_conj(t_from(be[i], T())) : t_from(ga[i], T());
            acc = t_add(acc, t_mul(sup, x[i + 1]));
        }
        y[i] = t_scale(acc, p);
    }
}

// <a, b> = sum conj(a_i) b_i over the block
template <typename T>
__device__ double2 bdot(int n, const T* a, const T* b, double2* sh) {
    double2 acc = mk(0.0, 0.0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc = cadd(acc, t_dotc(a[i], b[i]));
    return block_sum(acc, sh);
}

// a <- a - (u^dag a) u, u of unit norm (all threads of the block)
template <typename T>
__device__ void project_out(int n, const T* u, T* a, double2* sh) {
    double2 d = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) d = cadd(d, t_dotc(u[i], a[i]));
    d = block_sum(d, sh);
    const T dc = t_from(d, T());
    for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = t_sub(a[i], t_mul(dc, u[i]));
    __syncthreads();
}

// a Ritz pair counts as converged when its residual is at most this
// fraction of the Ritz value (p estimate)
constexpr double kPResidTol = 0.1;

template <typename T>
__device__ double bnorm(int n, const T* a, double* sh) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += t_norm2(a[i]);
    return sqrt(block_sum(acc, sh));
}

// ---- tridiagonal solves as warp-level scans of affine maps ---------------------
//
// The substitution sweeps of gttrs are linear recurrences.  A sequential chain
// leaves GB300's FP64 pipe 31/32 idle (a warp instruction with one active lane
// costs the pipe as much as a full one) and is latency bound, so each sweep
// runs on one warp as a parallel prefix over affine maps:
//   first order  (L sweep with interchanges):  s <- a s + c
//   second order (U sweep, two super-diagonals): X <- M X + v, X = (x_i, x_{i+1})
// Each lane composes the maps of its contiguous chunk, an exclusive shuffle
// scan composes the chunks before it, and the lane then walks its chunk from
// the state that scan gives.  The result is the LAPACK gttrs solution up to
// rounding order.  The U coefficients are precomputed once per LU:
//   x_i = e_i x_{i+1} + f_i x_{i+2} + y_i / d_i,   e_i = -du_i/d_i, f_i = -du2_i/d_i,
// and for the conjugate-transpose solve
//   x_i = eh_i x_{i-1} + fh_i x_{i-2} + b_i / d_i^*, eh_i = -(du_{i-1}/d_i)^*, fh_i = -(du2_{i-2}/d_i)^*.

constexpr unsigned kFull = 0xffffffffu;
__device__ __forceinline__ double shup(double v, int o) { return __shfl_up_sync(kFull, v, o); }
__device__ __forceinline__ double2 shup(double2 v, int o) {
    return mk(__shfl_up_sync(kFull, v.x, o), __shfl_up_sync(kFull, v.y, o));
}
__device__ __forceinline__ double shdn(double v, int o) { return __shfl_down_sync(kFull, v, o); }
__device__ __forceinline__ double2 shdn(double2 v, int o) {
    return mk(__shfl_down_sync(kFull, v.x, o), __shfl_down_sync(kFull, v.y, o));
}
__device__ __forceinline__ double t_one(double) { return 1.0; }
__device__ __forceinline__ double2 t_one(double2) { return mk(1.0, 0.0); }
// a * b + c
__device__ __forceinline__ double t_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double2 t_fma(double2 a, double2 b, double2 c) {
    return mk(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

template <typename T> struct Aff1 { T a, c; };                  // s -> a s + c
template <typename T> struct Aff2 { T m00, m01, m10, m11, v0, v1; };  // X -> M X + v

template <typename T> __device__ __forceinline__ Aff1<T> id1() { return {t_one(T()), t_zero(T())}; }
template <typename T> __device__ __forceinline__ Aff2<T> id2() {
    return {t_one(T()), t_zero(T()), t_zero(T()), t_one(T()), t_zero(T()), t_zero(T())};
}
// g o f (f applied first)
template <typename T> __device__ __forceinline__ Aff1<T> comp(const Aff1<T>& g, const Aff1<T>& f) {
    return {t_mul(g.a, f.a), t_fma(g.a, f.c, g.c)};
}
template <typename T> __device__ __forceinline__ Aff2<T> comp(const Aff2<T>& g, const Aff2<T>& f) {
    Aff2<T> r;
    r.m00 = t_fma(g.m00, f.m00, t_mul(g.m01, f.m10));
    r.m01 = t_fma(g.m00, f.m01, t_mul(g.m01, f.m11));
    r.m10 = t_fma(g.m10, f.m00, t_mul(g.m11, f.m10));
    r.m11 = t_fma(g.m10, f.m01, t_mul(g.m11, f.m11));
    r.v0 = t_fma(g.m00, f.v0, t_fma(g.m01, f.v1, g.v0));
    r.v1 = t_fma(g.m10, f.v0, t_fma(g.m11, f.v1, g.v1));
    return r;
}
template <typename T> __device__ __forceinline__ Aff1<T> shup(const Aff1<T>& f, int o) { return {shup(f.a, o), shup(f.c, o)}; }
template <typename T> __device__ __forceinline__ Aff1<T> shdn(const Aff1<T>& f, int o) { return {shdn(f.a, o), shdn(f.c, o)}; }
template <typename T> __device__ __forceinline__ Aff2<T> shup(const Aff2<T>& f, int o) {
    return {shup(f.m00, o), shup(f.m01, o), shup(f.m10, o), shup(f.m11, o), shup(f.v0, o), shup(f.v1, o)};
}
template <typename T> __device__ __forceinline__ Aff2<T> shdn(const Aff2<T>& f, int o) {
    return {shdn(f.m00, o), shdn(f.m01, o), shdn(f.m10, o), shdn(f.m11, o), shdn(f.v0, o), shdn(f.v1, o)};
}

// Exclusive scan over lanes: ascending (lower lanes' maps applied first) or
// descending (higher lanes' maps applied first).  Lane 0 (31) gets identity.
template <typename M> __device__ __forceinline__ M warp_exscan_up(M f, M ident) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        M p = shup(f, o);
        if (lane >= o) f = comp(f, p);
    }
    M ex = shup(f, 1);
    return lane == 0 ? ident : ex;
}
template <typename M> __device__ __forceinline__ M warp_exscan_down(M f, M ident) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        M p = shdn(f, o);
        if (lane + o < 32) f = comp(f, p);
    }
    M ex = shdn(f, 1);
    return lane == 31 ? ident : ex;
}

// Output of a sweep: plain store, or out = (out + x)/2 (the H' combination).
template <typename T> __device__ __forceinline__ void put(T* out, int i, T x, bool half_add) {
    out[i] = half_add ? t_scale(t_add(out[i], x), 0.5) : x;
}

// L sweep of (LU)^{-1}: y <- L^{-1} P b (forward, with the recorded interchanges).  in != out.
template <typename T>
__device__ void warp_L_fwd(int n, const T* __restrict__ dl, const int* __restrict__ ipiv,
                           const T* __restrict__ in, T* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int C = (n + 31) / 32;
    const int lo = min(lane * C, n), hi = min(lo + C, n);
    const int shi = min(hi, n - 1);   // steps i in [lo, shi)
    Aff1<T> F = id1<T>();
    for (int i = lo; i < shi; ++i) {
        const T bn = in[i + 1];
        Aff1<T> f = ipiv[i] == i ? Aff1<T>{t_scale(dl[i], -1.0), bn} : Aff1<T>{t_one(T()), t_scale(t_mul(dl[i], bn), -1.0)};
        F = comp(f, F);
    }
    const Aff1<T> G = warp_exscan_up(F, id1<T>());
    T st = t_fma(G.a, in[0], G.c);
    for (int i = lo; i < shi; ++i) {
        const T bn = in[i + 1];
        if (ipiv[i] == i) {
            out[i] = st;
            st = t_fma(t_scale(dl[i], -1.0), st, bn);
        } else {
            out[i] = bn;
            st = t_sub(st, t_mul(dl[i], bn));
        }
    }
    if (lo < hi && hi == n) out[n - 1] = st;
}

// U sweep: x_i = e_i x_{i+1} + f_i x_{i+2} + y_i dinv_i (descending).
template <typename T>
__device__ void warp_U_bwd(int n, const T* __restrict__ e, const T* __restrict__ f, const T* __restrict__ dinv,
                           const T* __restrict__ y, T* __restrict__ out, bool half_add) {
    const int lane = threadIdx.x & 31;
    const int C = (n + 31) / 32;
    const int lo = min(lane * C, n), hi = min(lo + C, n);
    Aff2<T> F = id2<T>();
    for (int i = hi - 1; i >= lo; --i) {
        Aff2<T> m = {e[i], f[i], t_one(T()), t_zero(T()), t_mul(y[i], dinv[i]), t_zero(T())};
        F = comp(m, F);
    }
    const Aff2<T> G = warp_exscan_down(F, id2<T>());
    T x1 = G.v0, x2 = G.v1;   // (x_{hi}, x_{hi+1})
    for (int i = hi - 1; i >= lo; --i) {
        const T x0 = t_fma(e[i], x1, t_fma(f[i], x2, t_mul(y[i], dinv[i])));
        put(out, i, x0, half_add);
        x2 = x1;
        x1 = x0;
    }
}

// U^dagger sweep: x_i = eh_i x_{i-1} + fh_i x_{i-2} + b_i conj(dinv_i) (ascending).  in != out.
template <typename T>
__device__ void warp_UH_fwd(int n, const T* __restrict__ eh, const T* __restrict__ fh, const T* __restrict__ dinv,
                            const T* __restrict__ in, T* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int C = (n + 31) / 32;
    const int lo = min(lane * C, n), hi = min(lo + C, n);
    Aff2<T> F = id2<T>();
    for (int i = lo; i < hi; ++i) {
        Aff2<T> m = {eh[i], fh[i], t_one(T()), t_zero(T()), t_mul(in[i], t_conj(dinv[i])), t_zero(T())};
        F = comp(m, F);
    }
    const Aff2<T> G = warp_exscan_up(F, id2<T>());
    T x1 = G.v0, x2 = G.v1;   // (x_{lo-1}, x_{lo-2})
    for (int i = lo; i < hi; ++i) {
        const T x0 = t_fma(eh[i], x1, t_fma(fh[i], x2, t_mul(in[i], t_conj(dinv[i]))));
        out[i] = x0;
        x2 = x1;
        x1 = x0;
    }
}

// L^dagger sweep of ((LU)^dagger)^{-1} (descending, interchanges undone).  in != out.
template <typename T>
__device__ void warp_LH_bwd(int n, const T* __restrict__ dl, const int* __restrict__ ipiv,
                            const T* __restrict__ in, T* __restrict__ out, bool half_add) {
    const int lane = threadIdx.x & 31;
    const int C = (n + 31) / 32;
    const int lo = min(lane * C, n), hi = min(lo + C, n);
    const int shi = min(hi, n - 1);   // steps i in [lo, shi), walked downwards
    Aff1<T> F = id1<T>();
    for (int i = shi - 1; i >= lo; --i) {
        Aff1<T> f = ipiv[i] == i ? Aff1<T>{t_scale(t_conj(dl[i]), -1.0), in[i]} : Aff1<T>{t_one(T()), t_zero(T())};
        F = comp(f, F);
    }
    const Aff1<T> G = warp_exscan_down(F, id1<T>());
    T st = t_fma(G.a, in[n - 1], G.c);   // s_{shi}: the value at position shi entering step shi - 1
    for (int i = shi - 1; i >= lo; --i) {
        const T cdl = t_conj(dl[i]);
        if (ipiv[i] == i) {
            put(out, i + 1, st, half_add);
            st = t_sub(in[i], t_mul(cdl, st));
        } else {
            put(out, i + 1, t_sub(in[i], t_mul(cdl, st)), half_add);
        }
    }
    if (lo == 0 && lo < hi) put(out, 0, st, half_add);
}

// After gttrf (which left du in e and du2 in f): the U coefficients of both
// solves.  All threads of the block.
template <typename T>
__device__ void lu_coefficients(int n, T* e, T* f, T* eh, T* fh, const T* dinv) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        eh[i] = i >= 1 ? t_scale(t_conj(t_mul(e[i - 1], dinv[i])), -1.0) : t_zero(T());
        fh[i] = i >= 2 ? t_scale(t_conj(t_mul(f[i - 2], dinv[i])), -1.0) : t_zero(T());
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        e[i] = i < n - 1 ? t_scale(t_mul(e[i], dinv[i]), -1.0) : t_zero(T());
        f[i] = i < n - 2 ? t_scale(t_mul(f[i], dinv[i]), -1.0) : t_zero(T());
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(256) k_inner(Inner in) {
    __shared__ double2 sh2[33];
    __shared__ double sh1[32];
    __shared__ int s_info;
    const int rhs = blockIdx.x;
    const int k = in.k, L = in.ell;
    if (in.status[rhs] != kStatusOK) return;
    const int ks = in.kstride > 0 ? in.kstride : k;   // row stride of the outer H_k arrays and of c
    const double2* al = in.alpha + (size_t)rhs * ks;
    const double2* be = in.beta + (size_t)rhs * ks;
    const double2* ga = in.gamma + (size_t)rhs * ks;
    // LU factors (in solve-ready form) and the two solve vectors in shared
    // memory.  While gttrf runs, d lives in t1, du in e and du2 in f.
    extern __shared__ __align__(16) unsigned char smem[];
    T* dl = reinterpret_cast<T*>(smem);
    T* dinv = dl + k;
    T* e = dinv + k;
    T* f = e + k;
    T* eh = f + k;
    T* fh = eh + k;
    T* t1 = fh + k;
    T* t2 = t1 + k;
    int* ipiv = reinterpret_cast<int*>(t2 + k);
    T* W = reinterpret_cast<T*>(in.work + (size_t)rhs * kInnerWorkVecs * k);
    T* x = W + 5 * (size_t)k;
    T* y = W + 6 * (size_t)k;
    T* vprev = W + 7 * (size_t)k;
    T* v = W + 8 * (size_t)k;
    T* r = W + 9 * (size_t)k;
    T* wprev = W + 10 * (size_t)k;
    T* w = W + 11 * (size_t)k;
    T* l = W + 12 * (size_t)k;
    const bool TS = sizeof(T) == sizeof(double2);
    const int warp = threadIdx.x >> 5;

    // LU of s * H in gttrf form, then the solve coefficients
    auto factor = [&](double sc) {
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            t1[i] = t_scale(t_from(al[i], T()), sc);
            if (i < k - 1) { dl[i] = t_scale(t_from(be[i], T()), sc); e[i] = t_scale(t_from(ga[i], T()), sc); }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_info = gttrf<T>(k, dl, t1, e, f, ipiv, dinv);
        __syncthreads();
        lu_coefficients<T>(k, e, f, eh, fh, dinv);
    };

    // ---- p (Eq. popt) --------------------------------------------------------
    double p = in.p_fixed;
    if (!(p > 0.0)) {
        const double x0 = 1.0 / sqrt((double)k);
        for (int i = threadIdx.x; i < k; i += blockDim.x) x[i] = t_from(mk(x0, 0.0), T());
        __syncthreads();
        double zmax = 0.0;
        for (int it = 0; it < 30; ++it) {
            band_mv<T>(k, 1.0, al, be, ga, x, y, false);
            __syncthreads();
            zmax = bnorm<T>(k, y, sh1);
            const double inv = 1.0 / zmax;
            for (int i = threadIdx.x; i < k; i += blockDim.x) x[i] = t_scale(y[i], inv);
            __syncthreads();
        }
        // inverse iteration with the LU of H itself
        factor(1.0);
        for (int i = threadIdx.x; i < k; i += blockDim.x) x[i] = t_from(mk(x0, 0.0), T());
        __syncthreads();
        double tn = 1.0;
        for (int it = 0; it < 30; ++it) {
            if (warp == 0) {
                warp_L_fwd<T>(k, dl, ipiv, x, t1);
                __syncwarp();
                warp_U_bwd<T>(k, e, f, dinv, t1, y, false);
            }
            __syncthreads();
            tn = bnorm<T>(k, y, sh1);
            const double inv = 1.0 / tn;
            for (int i = threadIdx.x; i < k; i += blockDim.x) x[i] = t_scale(y[i], inv);
            __syncthreads();
        }
        double zmin = 1.0 / tn;
        // Accept the smallest Ritz value only if its Ritz pair has converged
        // (residual |H(k-1,k-2)| |x_{k-1}| <= 0.1 z); otherwise it is a spurious
        // value in the spectral gap: iterate again with that direction projected out.
        const double resid = k >= 2 ? sqrt(cnorm2(be[k - 2])) * sqrt(t_norm2(x[k - 1])) : 0.0;
        if (resid > kPResidTol * zmin) {
            T* x1 = vprev;
            for (int i = threadIdx.x; i < k; i += blockDim.x) x1[i] = x[i];
            __syncthreads();
            for (int i = threadIdx.x; i < k; i += blockDim.x) x[i] = t_from(mk(x0, 0.0), T());
            __syncthreads();
            project_out<T>(k, x1, x, sh2);
            const double xn = bnorm<T>(k, x, sh1);
            for (int i = threadIdx.x; i < k; i += blockDim.x) x[i] = t_scale(x[i], 1.0 / xn);
            __syncthreads();
            for (int it = 0; it < 30; ++it) {
                if (warp == 0) {
                    warp_L_fwd<T>(k, dl, ipiv, x, t1);
                    __syncwarp();
                    warp_U_bwd<T>(k, e, f, dinv, t1, y, false);
                }
                __syncthreads();
                project_out<T>(k, x1, y, sh2);
                tn = bnorm<T>(k, y, sh1);
                const double inv = 1.0 / tn;
                for (int i = threadIdx.x; i < k; i += blockDim.x) x[i] = t_scale(y[i], inv);
                __syncthreads();
            }
            zmin = 1.0 / tn;
        }
        p = 1.0 / sqrt(zmin * zmax);
        if (threadIdx.x == 0) { in.zmin[rhs] = zmin; in.zmax[rhs] = zmax; }
    } else if (threadIdx.x == 0) {
        in.zmin[rhs] = 0.0; in.zmax[rhs] = 0.0;
    }
    if (threadIdx.x == 0) in.p[rhs] = p;

    // ---- step 3: LU of p H_k --------------------------------------------------
    factor(p);
    if (s_info != 0) {
        if (threadIdx.x == 0) in.status[rhs] = kStatusLU;
        return;
    }

    // ---- step 4: inner (two-sided) Lanczos with H' and e_1 ----------------------
    // H' x = [(pH) x + (pH)^{-1} x] / 2 into out; with dagger for the left recurrence.
    double2* Vl = in.Vl + (size_t)rhs * L * k;
    auto store_vl = [&](int j, const T* src) {
        for (int i = threadIdx.x; i < k; i += blockDim.x) Vl[(size_t)j * k + i] = t_to2(src[i]);
    };
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        v[i] = t_zero(T());
        if (TS) w[i] = t_zero(T());
    }
    __syncthreads();
    if (threadIdx.x == 0) { v[0] = t_from(mk(1.0, 0.0), T()); if (TS) w[0] = v[0]; }
    __syncthreads();
    store_vl(0, v);

    // out_r = H' src_r = [(pH) src_r + (pH)^{-1} src_r]/2 and, two-sided,
    // out_l = H'^dagger src_l: band products by the whole block, then the
    // (pH)^{-1} solve on warp 0 and the ((pH)^dagger)^{-1} solve on warp 1.
    auto apply_hp = [&](const T* src_r, T* out_r, const T* src_l, T* out_l) {
        band_mv<T>(k, p, al, be, ga, src_r, out_r, false);
        if (TS) band_mv<T>(k, p, al, be, ga, src_l, out_l, true);
        __syncthreads();
        if (warp == 0) {
            warp_L_fwd<T>(k, dl, ipiv, src_r, t1);
            __syncwarp();
            warp_U_bwd<T>(k, e, f, dinv, t1, out_r, true);
        } else if (TS && warp == 1) {
            warp_UH_fwd<T>(k, eh, fh, dinv, src_l, t2);
            __syncwarp();
            warp_LH_bwd<T>(k, dl, ipiv, t2, out_l, true);
        }
        __syncthreads();
    };

    apply_hp(v, r, w, l);  // r <- H' v_1, l <- H'^dag w_1
    double2* alo = in.al + (size_t)rhs * L;
    double2* blo = in.bl + (size_t)rhs * L;
    double2* glo = in.gl + (size_t)rhs * L;
    for (int j = 0; j < L; ++j) {
        // H(j,j) <- v^dag r (two-sided: w^dag r)
        double2 a2 = bdot<T>(k, TS ? w : v, r, sh2);
        T a = TS ? t_from(a2, T()) : t_from(mk(a2.x, 0.0), T());
        if (threadIdx.x == 0) alo[j] = t_to2(a);
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            r[i] = t_sub(r[i], t_mul(a, v[i]));
            if (TS) l[i] = t_sub(l[i], t_mul(t_conj(a), w[i]));
        }
        __syncthreads();
        if (j == L - 1) break;
        T bb, gg;
        if (!TS) {
            double b = bnorm<T>(k, r, sh1);            // beta <- |r|
            bb = t_from(mk(b, 0.0), T());
            gg = bb;
            if (!(b > 0.0)) { if (threadIdx.x == 0) in.status[rhs] = kStatusBreakdown; return; }
        } else {
            double2 dlt = bdot<T>(k, r, l, sh2);        // delta <- r^dag l
            if ((dlt.x == 0.0 && dlt.y == 0.0) || !isfinite(dlt.x) || !isfinite(dlt.y)) {
                if (threadIdx.x == 0) in.status[rhs] = kStatusBreakdown;
                return;
            }
            double2 b2 = csqrt_principal(dlt);
            bb = t_from(b2, T());
            gg = t_from(cdiv(cconj(dlt), b2), T());
        }
        if (threadIdx.x == 0) { blo[j] = t_to2(bb); glo[j] = t_to2(gg); }
        const T binv = t_inv(bb);
        const T ginv = t_inv(t_conj(gg));
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            vprev[i] = v[i];
            v[i] = t_mul(r[i], binv);                   // v <- r / beta
            if (TS) { wprev[i] = w[i]; w[i] = t_mul(l[i], ginv); }   // w <- l / gamma^*
        }
        __syncthreads();
        store_vl(j + 1, v);
        apply_hp(v, r, w, l);
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            r[i] = t_sub(r[i], t_mul(gg, vprev[i]));    // r <- r - gamma v_j
            if (TS) l[i] = t_sub(l[i], t_mul(t_conj(bb), wprev[i]));   // l <- l - beta^* w_j
        }
        __syncthreads();
    }
}

// ---- Roberts-Higham iteration on H_l, one cluster per RHS ----------------------

constexpr int kRhiThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kRhiThreads) k_rhi(Inner in, int C, int maxit, double stop) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int rhs = blockIdx.x / C;
    const int L = in.ell;
    const int nloc = (L - rank + C - 1) / C;       // rows rank, rank + C, ...
    const int nmax = (L + C - 1) / C;
    extern __shared__ __align__(16) unsigned char smem[];
    T* M = reinterpret_cast<T*>(smem);              // [nmax][L]
    T* prow = M + (size_t)nmax * L;                 // [L]
    T* tmp = prow + L;                              // [L]
    T* fcol = tmp + L;                              // [nmax]
    int* piv = reinterpret_cast<int*>(fcol + nmax); // [L]
    __shared__ double cand_val;
    __shared__ int cand_idx;
    __shared__ double part[2];
    __shared__ double red_v[kRhiThreads / 32];
    __shared__ int red_i[kRhiThreads / 32];
    __shared__ double sh1[32];
    __shared__ int s_stop;

    const int status0 = in.status[rhs];   // identical in every CTA of the cluster
    T* S = reinterpret_cast<T*>(in.S) + (size_t)rhs * L * L;
    const double2* alo = in.al + (size_t)rhs * L;
    const double2* blo = in.bl + (size_t)rhs * L;
    const double2* glo = in.gl + (size_t)rhs * L;
    const int tid = threadIdx.x;

    // S_0 = H_l (own rows)
    for (int e = tid; e < nloc * L; e += blockDim.x) {
        int li = e / L, col = e % L, i = rank + C * li;
        T v = t_zero(T());
        if (status0 == kStatusOK) {
            if (col == i) v = t_from(alo[i], T());
            else if (col == i - 1) v = t_from(blo[i - 1], T());
            else if (col == i + 1) v = t_from(glo[i], T());
        }
        S[(size_t)i * L + col] = v;
    }
    int iters = 0;
    bool ok = status0 == kStatusOK;
    bool converged = false;
    for (int it = 1; ok && it <= maxit; ++it) {
        iters = it;
        for (int e = tid; e < nloc * L; e += blockDim.x) {
            int li = e / L, col = e % L;
            M[(size_t)li * L + col] = S[(size_t)(rank + C * li) * L + col];
        }
        __syncthreads();
        // ---- in-place Gauss-Jordan inverse of M with partial pivoting ----
        for (int c = 0; c < L; ++c) {
            // (a) local candidate: largest |M(i,c)|^2 over own rows i >= c (lowest i on ties)
            double bv = -1.0;
            int bi = 0x7fffffff;
            for (int li = tid; li < nloc; li += blockDim.x) {
                int i = rank + C * li;
                if (i < c) continue;
                double m = t_norm2(M[(size_t)li * L + c]);
                if (m > bv || (m == bv && i < bi)) { bv = m; bi = i; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            if ((tid & 31) == 0) { red_v[tid >> 5] = bv; red_i[tid >> 5] = bi; }
            __syncthreads();
            if (tid == 0) {
                for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
                    if (red_v[q] > bv || (red_v[q] == bv && red_i[q] < bi)) { bv = red_v[q]; bi = red_i[q]; }
                cand_val = bv;
                cand_idx = bi;
            }
            cl.sync();                                                  // barrier A
            // (b) pivot row over the cluster, ranks in fixed order
            double pv = -1.0;
            int pi = 0x7fffffff;
            for (int q = 0; q < C; ++q) {
                double qv = *cl.map_shared_rank(&cand_val, q);
                int qi = *cl.map_shared_rank(&cand_idx, q);
                if (qv > pv || (qv == pv && qi < pi)) { pv = qv; pi = qi; }
            }
            if (!(pv > 0.0)) {              // singular (same decision in every CTA)
                ok = false;
                cl.sync();
                break;
            }
            if (tid == 0) piv[c] = pi;
            // (c) fetch the pivot row (and, for its owner, old row c)
            {
                T* src = cl.map_shared_rank(M, pi % C) + (size_t)(pi / C) * L;
                for (int col = tid; col < L; col += blockDim.x) prow[col] = src[col];
                if (pi != c && pi % C == rank) {
                    T* srcc = cl.map_shared_rank(M, c % C) + (size_t)(c / C) * L;
                    for (int col = tid; col < L; col += blockDim.x) tmp[col] = srcc[col];
                }
            }
            cl.sync();                                                  // barrier B
            // (d) interchange and scale the pivot row
            if (pi != c && pi % C == rank) {
                T* dst = M + (size_t)(pi / C) * L;
                for (int col = tid; col < L; col += blockDim.x) dst[col] = tmp[col];
            }
            const T pinv = t_inv(prow[c]);
            __syncthreads();
            for (int col = tid; col < L; col += blockDim.x)
                if (col != c) prow[col] = t_mul(prow[col], pinv);
            __syncthreads();
            if (tid == 0) prow[c] = pinv;
            __syncthreads();
            if (c % C == rank) {
                T* dst = M + (size_t)(c / C) * L;
                for (int col = tid; col < L; col += blockDim.x) dst[col] = prow[col];
            }
            // (e) eliminate column c from every other own row: M(i,:) -= M(i,c) prow,
            // then M(i,c) = -M(i,c) pinv (the multipliers, read first)
            for (int li = tid; li < nloc; li += blockDim.x) fcol[li] = M[(size_t)li * L + c];
            __syncthreads();
            for (int e = tid; e < nloc * L; e += blockDim.x) {
                const int li = e / L, col = e % L;
                if (rank + C * li == c || col == c) continue;
                T& m = M[(size_t)li * L + col];
                m = t_fma(t_neg(fcol[li]), prow[col], m);
            }
            for (int li = tid; li < nloc; li += blockDim.x)
                if (rank + C * li != c) M[(size_t)li * L + c] = t_mul(t_neg(fcol[li]), pinv);
            __syncthreads();
        }
        if (!ok) break;
        // undo the interchanges on the columns of the inverse
        for (int c = L - 1; c >= 0; --c) {
            int q = piv[c];
            if (q != c) {
                for (int li = tid; li < nloc; li += blockDim.x) {
                    T a = M[(size_t)li * L + c];
                    M[(size_t)li * L + c] = M[(size_t)li * L + q];
                    M[(size_t)li * L + q] = a;
                }
            }
            __syncthreads();
        }
        // S <- (S + S^{-1}) / 2 and the relative Frobenius change
        double dsum = 0.0, nsum = 0.0;
        for (int e = tid; e < nloc * L; e += blockDim.x) {
            int li = e / L, col = e % L;
            size_t gi = (size_t)(rank + C * li) * L + col;
            T so = S[gi];
            T sn = t_scale(t_add(so, M[(size_t)li * L + col]), 0.5);
            dsum += t_norm2(t_sub(sn, so));
            nsum += t_norm2(sn);
            S[gi] = sn;
        }
        dsum = block_sum(dsum, sh1);
        nsum = block_sum(nsum, sh1);
        if (tid == 0) { part[0] = dsum; part[1] = nsum; }
        cl.sync();
        double dt = 0.0, nt = 0.0;
        for (int q = 0; q < C; ++q) {
            const double* pq = cl.map_shared_rank(part, q);
            dt += pq[0];
            nt += pq[1];
        }
        cl.sync();   // every CTA has read the partials before they are rewritten
        if (sqrt(dt) <= stop * sqrt(nt)) { converged = true; break; }
    }
    if (tid == 0) s_stop = 0;
    __syncthreads();
    // s = S e_1 (own rows), iteration count, status
    for (int li = tid; li < nloc; li += blockDim.x) {
        int i = rank + C * li;
        in.s[(size_t)rhs * L + i] = t_to2(S[(size_t)i * L]);
    }
    if (rank == 0 && tid == 0) {
        in.rhi_iters[rhs] = iters;
        if (status0 == kStatusOK && !converged) in.status[rhs] = kStatusRhi;
    }
}

// c = V_l s (k-vector per RHS)
__global__ void k_combine(Inner in) {
    const int rhs = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= in.k) return;
    double2* c = in.c + (size_t)rhs * (in.kstride > 0 ? in.kstride : in.k);
    if (in.status[rhs] != kStatusOK) { c[i] = mk(0.0, 0.0); return; }
    const double2* Vl = in.Vl + (size_t)rhs * in.ell * in.k;
    const double2* s = in.s + (size_t)rhs * in.ell;
    double2 acc = mk(0.0, 0.0);
    for (int j = 0; j < in.ell; ++j) acc = cadd(acc, cmul(Vl[(size_t)j * in.k + i], s[j]));
    c[i] = acc;
}

}  // namespace

size_t inner_smem_bytes(int k, bool two_sided) {
    return (size_t)k * (8 * (two_sided ? sizeof(double2) : sizeof(double)) + sizeof(int));
}

void launch_inner_lanczos(const Inner& in, cudaStream_t st) {
    size_t smem = inner_smem_bytes(in.k, in.two_sided);
    if (in.two_sided) k_inner<double2><<<in.n_rhs, 256, smem, st>>>(in);
    else k_inner<double><<<in.n_rhs, 256, smem, st>>>(in);
}

// Largest dynamic shared memory any RHi launch needs (l <= 256, complex, 8 CTAs).
static size_t rhi_smem_max();
size_t inner_smem_bytes(int k, bool two_sided);

void init_kernel_attributes() {
    cudaFuncSetAttribute(k_inner<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)inner_smem_bytes(kMaxInnerK, false));
    cudaFuncSetAttribute(k_inner<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)inner_smem_bytes(kMaxInnerK, true));
    cudaFuncSetAttribute(k_rhi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhi_smem_max());
    cudaFuncSetAttribute(k_rhi<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhi_smem_max());
    cudaFuncSetAttribute(k_rhi<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_rhi<double2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

static int rhi_cluster_size(int ell) { return ell >= 64 ? 8 : (ell >= 16 ? 4 : 1); }

template <typename T>
static size_t rhi_smem(int ell, int C) {
    int nmax = (ell + C - 1) / C;
    return (size_t)nmax * ell * sizeof(T) + 2 * (size_t)ell * sizeof(T) + (size_t)nmax * sizeof(T) +
           (size_t)ell * sizeof(int) + 16;
}

static size_t rhi_smem_max() { return rhi_smem<double2>(256, 8); }

template <typename T>
static cudaError_t launch_rhi_t(const Inner& in, cudaStream_t st) {
    const int C = rhi_cluster_size(in.ell);
    size_t smem = rhi_smem<T>(in.ell, C);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(in.n_rhs * C);
    cfg.blockDim = dim3(kRhiThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_rhi<T>, in, C, 50, 1e-10);
}

int launch_rhi(const Inner& in, cudaStream_t st) {
    return (int)(in.two_sided ? launch_rhi_t<double2>(in, st) : launch_rhi_t<double>(in, st));
}

void launch_inner_combine(const Inner& in, cudaStream_t st) {
    dim3 grid((in.k + 127) / 128, in.n_rhs);
    k_combine<<<grid, 128, 0, st>>>(in);
}

}  // namespace nk
