// Inner half of the nested method, per RHS (App. C steps 3-5, Eqs. popt,
// precond, innersign, Roberts):
//   p      = (z_min z_max)^{-1/2}, z_max by power iteration with H_k and z_min
//            by inverse iteration with the LU of H_k (30 steps each, from the
//            normalised all-ones vector), unless p is given; with one p for
//            the batch, z_min and z_max are the extremes over its RHS (two
//            launches: the estimates of every RHS, then the rest);
//   LU of p H_k in LAPACK gttrf form (partial pivoting; U with two super-diagonals);
//   inner (two-sided) Lanczos of size l with H_k' = [p H_k + (p H_k)^{-1}]/2 and
//            e_1, applying (p H_k)^{-1} by the gttrs back substitution and
//            p H_k by a band product (App. C step 4 (a), (b));
//   Roberts-Higham iteration S <- (S + S^{-1})/2 on the dense H_l;
//   c = V_l sgn(H_l) e_1.
// In the Hermitian case (mu = 0) all of it is real arithmetic (App. C).
//
// The inner Lanczos runs one CTA per RHS: the band products, inner products
// and axpys are spread over the CTA; the two O(k) substitution sweeps of each
// solve are parallel prefix scans on a group of 4 warps (two groups in the
// two-sided case, where H_k' v and H_k'^dagger w are independent),
// with the parts of the scans that depend on the LU factors alone tabulated
// once per LU.
//
// RHi runs one thread-block cluster per RHS: the rows of the l x l matrix
// being inverted (in-place Gauss-Jordan with partial pivoting and row
// interchanges) are spread cyclically over the cluster's CTAs and held in
// their shared memory; the pivot search, the pivot row broadcast and the row
// interchange go through distributed shared memory, with one cluster barrier
// per pivot (candidate rows published in buffers that alternate between
// pivots).
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

// ---- the same on T = df (real) or dfc (complex): two-float arithmetic on the
// FP32 pipe, for the inner part of the mixed schedule ---------------------------
__device__ __forceinline__ df t_zero(df) { return df(0); }
__device__ __forceinline__ dfc t_zero(dfc) { dfc r; r.x = df(0); r.y = df(0); return r; }
__device__ __forceinline__ df t_from(double2 a, df) { return df_from_double(a.x); }
__device__ __forceinline__ dfc t_from(double2 a, dfc) { dfc r; r.x = df_from_double(a.x); r.y = df_from_double(a.y); return r; }
__device__ __forceinline__ double2 t_to2(df a) { return mk(df_to_double(a), 0.0); }
__device__ __forceinline__ double2 t_to2(dfc a) { return mk(df_to_double(a.x), df_to_double(a.y)); }
__device__ __forceinline__ df t_conj(df a) { return a; }
__device__ __forceinline__ dfc t_conj(dfc a) { dfc r; r.x = a.x; r.y = -a.y; return r; }
__device__ __forceinline__ df t_mul(df a, df b) { return a * b; }
__device__ __forceinline__ dfc t_mul(dfc a, dfc b) {
    dfc r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
__device__ __forceinline__ df t_add(df a, df b) { return a + b; }
__device__ __forceinline__ dfc t_add(dfc a, dfc b) { dfc r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
__device__ __forceinline__ df t_sub(df a, df b) { return a - b; }
__device__ __forceinline__ dfc t_sub(dfc a, dfc b) { dfc r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// scaling by -1 and 1/2 is exact; other factors go through a two-float product
__device__ __forceinline__ df t_scale(df a, double s) {
    if (s == -1.0) return -a;
    if (s == 0.5) return df(a.hi * 0.5f, a.lo * 0.5f);
    return a * df_from_double(s);
}
__device__ __forceinline__ dfc t_scale(dfc a, double s) { dfc r; r.x = t_scale(a.x, s); r.y = t_scale(a.y, s); return r; }
__device__ __forceinline__ df t_neg(df a) { return -a; }
__device__ __forceinline__ dfc t_neg(dfc a) { dfc r; r.x = -a.x; r.y = -a.y; return r; }
// 1/a: the FP32 reciprocal refined by one Newton step in two-float arithmetic
__device__ __forceinline__ df t_inv(df a) {
    const df y0(__frcp_rn(a.hi), 0.0f);
    const df e = df(1) - a * y0;
    return y0 + y0 * e;
}
__device__ __forceinline__ dfc t_inv(dfc a) {
    const df ninv = t_inv(a.x * a.x + a.y * a.y);
    dfc r;
    r.x = a.x * ninv;
    r.y = -(a.y * ninv);
    return r;
}
// pivot magnitudes (gttrf's choice only): from the high parts
__device__ __forceinline__ double t_abs1(df a) { return fabsf(a.hi); }
__device__ __forceinline__ double t_abs1(dfc a) { return fabsf(a.x.hi) + fabsf(a.y.hi); }
__device__ __forceinline__ double t_norm2(df a) { return df_to_double(a * a); }
__device__ __forceinline__ double t_norm2(dfc a) { return df_to_double(a.x * a.x + a.y * a.y); }
__device__ __forceinline__ bool t_iszero(df a) { return a.hi == 0.0f && a.lo == 0.0f; }
__device__ __forceinline__ bool t_iszero(dfc a) { return t_iszero(a.x) && t_iszero(a.y); }
__device__ __forceinline__ double2 t_dotc(df a, df b) { return mk(df_to_double(a * b), 0.0); }
__device__ __forceinline__ double2 t_dotc(dfc a, dfc b) {
    return mk(df_to_double(a.x * b.x + a.y * b.y), df_to_double(a.x * b.y - a.y * b.x));
}
template <typename T> struct IsDF { static constexpr bool value = false; };
template <> struct IsDF<df> { static constexpr bool value = true; };
template <> struct IsDF<dfc> { static constexpr bool value = true; };
// two-float partial sums of conj(a) b and |a|^2, converted once per thread
__device__ __forceinline__ void dotc_acc(df a, df b, df& sx, df&) { sx += a * b; }
__device__ __forceinline__ void dotc_acc(dfc a, dfc b, df& sx, df& sy) {
    sx += a.x * b.x + a.y * b.y;
    sy += a.x * b.y - a.y * b.x;
}
__device__ __forceinline__ df norm2_df(df a) { return a * a; }
__device__ __forceinline__ df norm2_df(dfc a) { return a.x * a.x + a.y * a.y; }

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
// summation order (diag, sub, super) -- all threads of the block.  The
// diagonals come as T arrays (converted once per kernel).
template <typename T>
__device__ void band_mv(int n, double p, const T* al, const T* be, const T* ga,
                        const T* x, T* y, bool dagger) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        T dg = al[i];
        if (dagger) dg = t_conj(dg);
        T acc = t_mul(dg, x[i]);
        if (i > 0) {
            T sub = dagger ? t_conj(ga[i - 1]) : be[i - 1];
            acc = t_add(acc, t_mul(sub, x[i - 1]));
        }
        if (i < n - 1) {
            T sup = dagger ? t_conj(be[i]) : ga[i];
            acc = t_add(acc, t_mul(sup, x[i + 1]));
        }
        y[i] = t_scale(acc, p);
    }
}

// <a, b> = sum conj(a_i) b_i over the block
template <typename T>
__device__ double2 bdot(int n, const T* a, const T* b, double2* sh) {
    double2 acc = mk(0.0, 0.0);
    if constexpr (IsDF<T>::value) {
        df sx(0), sy(0);
        for (int i = threadIdx.x; i < n; i += blockDim.x) dotc_acc(a[i], b[i], sx, sy);
        acc = mk(df_to_double(sx), df_to_double(sy));
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) acc = cadd(acc, t_dotc(a[i], b[i]));
    }
    return block_sum(acc, sh);
}

// a <- a - (u^dag a) u, u of unit norm (all threads of the block)
template <typename T>
__device__ void project_out(int n, const T* u, T* a, double2* sh) {
    double2 d = bdot<T>(n, u, a, sh);
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
    if constexpr (IsDF<T>::value) {
        df sx(0);
        for (int i = threadIdx.x; i < n; i += blockDim.x) sx += norm2_df(a[i]);
        acc = df_to_double(sx);
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) acc += t_norm2(a[i]);
    }
    return sqrt(block_sum(acc, sh));
}

// ---- tridiagonal solves as scans of affine maps ---------------------------------
//
// The substitution sweeps of gttrs are linear recurrences.  A sequential chain
// leaves GB300's FP64 pipe 31/32 idle (a warp instruction with one active lane
// costs the pipe as much as a full one) and is latency bound, so each sweep
// runs as a parallel prefix over affine maps:
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
__device__ __forceinline__ df shup(df v, int o) { return df(__shfl_up_sync(kFull, v.hi, o), __shfl_up_sync(kFull, v.lo, o)); }
__device__ __forceinline__ df shdn(df v, int o) { return df(__shfl_down_sync(kFull, v.hi, o), __shfl_down_sync(kFull, v.lo, o)); }
__device__ __forceinline__ dfc shup(dfc v, int o) { dfc r; r.x = shup(v.x, o); r.y = shup(v.y, o); return r; }
__device__ __forceinline__ dfc shdn(dfc v, int o) { dfc r; r.x = shdn(v.x, o); r.y = shdn(v.y, o); return r; }
__device__ __forceinline__ df t_one(df) { return df(1); }
__device__ __forceinline__ dfc t_one(dfc) { dfc r; r.x = df(1); r.y = df(0); return r; }
__device__ __forceinline__ df t_fma(df a, df b, df c) { return a * b + c; }
__device__ __forceinline__ dfc t_fma(dfc a, dfc b, dfc c) { return t_add(t_mul(a, b), c); }

// The maps of a sweep split into a part that depends on the LU factors only
// (a of s <- a s + c; M of X <- M X + v) and a part that depends on the
// right-hand side (c; v).  The factor parts are composed once per LU
// (sweep_tables) and kept in a per-RHS table; a solve then composes only the
// right-hand-side parts: first order 1 complex product per element, second
// order 3 (the companion matrix [[e, f], [1, 0]] is sparse).
// Composition rules (g after f):
//   first order   (a, c): a = a_g a_f,  c = a_g c_f + c_g;
//   second order  (M, v): M = M_g M_f,  v = M_g v_f + v_g.
//
// A solve runs on a group of W = 4 warps (warps 0-3; in the two-sided case
// warps 4-7 solve with H'^dagger side by side), so all four SM sub-partitions
// issue its FP64 work.  Each of the 32 W lanes takes a contiguous chunk; the
// chunk maps are composed by a shuffle scan inside each warp and by a short
// sequential composition of the W warp aggregates (exchanged through shared
// memory between two group barriers).  Positions run in the order the maps
// are applied: ascending sweeps from chunk 0, descending ones from the last.
//
// Table rows ([row][group lane], NL = 32 W lanes per row):
//   first order:  0-4 a before each shuffle level, 5 a of the intra-warp
//                 exclusive prefix, 6 a of the whole exclusive prefix,
//                 7 a of each warp's aggregate (indexed by warp position);
//   second order: 0-19 M before each level (4 entries per level), 20-23 M of
//                 the intra-warp exclusive prefix, 24-27 M of each warp's
//                 aggregate (indexed by warp position).
constexpr int kRowsFirst = 8, kRowsSecond = 28;
constexpr int kTabL = 0, kTabLH = kRowsFirst, kTabU = 2 * kRowsFirst, kTabUH = 2 * kRowsFirst + kRowsSecond;
constexpr int kTabRows = 2 * kRowsFirst + 2 * kRowsSecond;
static_assert(kTabRows * 256 <= kSweepTableElems, "sweep tables do not fit the work area");

// The warp group of the calling thread.  Group g uses named barrier 1 + g.
struct Grp {
    int W;      // warps in the group
    int gw;     // this warp's index in the group
    int lane;
    int bar;    // named barrier id
    int g;      // group index
};
__device__ __forceinline__ Grp grp_of(bool) {
    const int warp = threadIdx.x >> 5;
    const int W = 4;
    return {W, warp % W, (int)(threadIdx.x & 31), 1 + warp / W, warp / W};
}
__device__ __forceinline__ void grp_sync(const Grp& G) {
    asm volatile("bar.sync %0, %1;" ::"r"(G.bar), "r"(G.W * 32) : "memory");
}
// chunk [lo, hi) of group lane gw*32 + lane over n elements
__device__ __forceinline__ void grp_chunk(const Grp& G, int n, int& lo, int& hi) {
    const int NL = 32 * G.W;
    const int C = (n + NL - 1) / NL;
    lo = min((G.gw * 32 + G.lane) * C, n);
    hi = min(lo + C, n);
}

template <typename T> struct Mat2 { T m00, m01, m10, m11; };
template <typename T> __device__ __forceinline__ Mat2<T> mat_mul(const Mat2<T>& g, const Mat2<T>& f) {
    return {t_fma(g.m00, f.m00, t_mul(g.m01, f.m10)), t_fma(g.m00, f.m01, t_mul(g.m01, f.m11)),
            t_fma(g.m10, f.m00, t_mul(g.m11, f.m10)), t_fma(g.m10, f.m01, t_mul(g.m11, f.m11))};
}
template <typename T> __device__ __forceinline__ T shfl_dir(T v, int o, bool asc) { return asc ? shup(v, o) : shdn(v, o); }
template <typename T> __device__ __forceinline__ Mat2<T> shfl_mat(const Mat2<T>& a, int o, bool asc) {
    return {shfl_dir(a.m00, o, asc), shfl_dir(a.m01, o, asc), shfl_dir(a.m10, o, asc), shfl_dir(a.m11, o, asc)};
}
template <typename T> __device__ __forceinline__ T shfl_from(T v, int src) {
    return t_from(mk(__shfl_sync(kFull, t_to2(v).x, src), __shfl_sync(kFull, t_to2(v).y, src)), T());
}
__device__ __forceinline__ double shfl_from(double v, int src) { return __shfl_sync(kFull, v, src); }
// partner exists at shuffle distance o; first / last position lanes
__device__ __forceinline__ bool has_partner(int lane, int o, bool asc) { return asc ? lane >= o : lane + o < 32; }
__device__ __forceinline__ int last_lane(bool asc) { return asc ? 31 : 0; }
__device__ __forceinline__ bool first_lane(int lane, bool asc) { return asc ? lane == 0 : lane == 31; }
__device__ __forceinline__ int warp_pos(const Grp& G, bool asc) { return asc ? G.gw : G.W - 1 - G.gw; }

// first-order factor table (a_i = -dl_i, or -conj(dl_i) for the dagger sweep,
// where row i was not interchanged, 1 where it was); all warps of the group
template <typename T>
__device__ void table_first_order(const Grp& G, int n, const T* __restrict__ dl, const int* __restrict__ ipiv,
                                  bool dagger, T* tab, double2* s_agg) {
    const int NL = 32 * G.W, gl = G.gw * 32 + G.lane;
    const bool asc = !dagger;
    int lo, hi;
    grp_chunk(G, n, lo, hi);
    const int shi = min(hi, n - 1);
    T A = t_one(T());
    for (int i = lo; i < shi; ++i)
        if (ipiv[i] == i) A = t_mul(t_scale(dagger ? t_conj(dl[i]) : dl[i], -1.0), A);
    for (int lv = 0, o = 1; o < 32; ++lv, o <<= 1) {
        tab[lv * NL + gl] = A;
        const T pa = shfl_dir(A, o, asc);
        if (has_partner(G.lane, o, asc)) A = t_mul(A, pa);
    }
    const T ex = shfl_dir(A, 1, asc);
    const T a_ex = first_lane(G.lane, asc) ? t_one(T()) : ex;
    tab[5 * NL + gl] = a_ex;
    const T agg = shfl_from(A, last_lane(asc));
    const int pw = warp_pos(G, asc);
    if (G.lane == 0) { tab[7 * NL + pw] = agg; s_agg[G.gw] = t_to2(agg); }
    grp_sync(G);
    T P = t_one(T());
    for (int q = 0; q < G.W; ++q) {
        const int qw = asc ? q : G.W - 1 - q;    // group warp at position q
        if (q < pw) P = t_mul(t_from(s_agg[qw], T()), P);
    }
    tab[6 * NL + gl] = t_mul(a_ex, P);
    grp_sync(G);
}

// second-order factor table: M_i = [[e_i, f_i], [1, 0]] (descending for U,
// ascending for U^dagger); all warps of the group
template <typename T>
__device__ void table_second_order(const Grp& G, int n, const T* __restrict__ e, const T* __restrict__ f, bool asc,
                                   T* tab) {
    const int NL = 32 * G.W, gl = G.gw * 32 + G.lane;
    int lo, hi;
    grp_chunk(G, n, lo, hi);
    Mat2<T> F = {t_one(T()), t_zero(T()), t_zero(T()), t_one(T())};
    auto step = [&](int i) {
        F = {t_fma(e[i], F.m00, t_mul(f[i], F.m10)), t_fma(e[i], F.m01, t_mul(f[i], F.m11)), F.m00, F.m01};
    };
    if (asc) for (int i = lo; i < hi; ++i) step(i);
    else for (int i = hi - 1; i >= lo; --i) step(i);
    for (int lv = 0, o = 1; o < 32; ++lv, o <<= 1) {
        tab[(4 * lv + 0) * NL + gl] = F.m00;
        tab[(4 * lv + 1) * NL + gl] = F.m01;
        tab[(4 * lv + 2) * NL + gl] = F.m10;
        tab[(4 * lv + 3) * NL + gl] = F.m11;
        const Mat2<T> Pm = shfl_mat(F, o, asc);
        if (has_partner(G.lane, o, asc)) F = mat_mul(F, Pm);
    }
    const Mat2<T> ex = shfl_mat(F, 1, asc);
    const bool first = first_lane(G.lane, asc);
    tab[20 * NL + gl] = first ? t_one(T()) : ex.m00;
    tab[21 * NL + gl] = first ? t_zero(T()) : ex.m01;
    tab[22 * NL + gl] = first ? t_zero(T()) : ex.m10;
    tab[23 * NL + gl] = first ? t_one(T()) : ex.m11;
    const int ll = last_lane(asc);
    const T a00 = shfl_from(F.m00, ll), a01 = shfl_from(F.m01, ll);
    const T a10 = shfl_from(F.m10, ll), a11 = shfl_from(F.m11, ll);
    if (G.lane == 0) {
        const int pw = warp_pos(G, asc);
        tab[24 * NL + pw] = a00;
        tab[25 * NL + pw] = a01;
        tab[26 * NL + pw] = a10;
        tab[27 * NL + pw] = a11;
    }
}

// The tables of one LU.  Hermitian: the one group builds L then U; two-sided:
// group 0 builds L and U, group 1 the dagger sweeps.  Ends with a block barrier.
template <typename T>
__device__ void sweep_tables(int n, const T* dl, const int* ipiv, const T* e, const T* f, const T* eh,
                             const T* fh, bool two_sided, T* tab, double2* s_agg) {
    const Grp G = grp_of(two_sided);
    const int NL = 32 * G.W;
    double2* agg = s_agg + 16 * G.g;
    if (G.g == 0) {
        table_first_order<T>(G, n, dl, ipiv, false, tab + kTabL * NL, agg);
        table_second_order<T>(G, n, e, f, false, tab + kTabU * NL);
    } else if (two_sided) {
        table_first_order<T>(G, n, dl, ipiv, true, tab + kTabLH * NL, agg);
        table_second_order<T>(G, n, eh, fh, true, tab + kTabUH * NL);
    }
    __syncthreads();
}

// intra-warp inclusive scans of right-hand-side parts with tabulated factor parts
template <typename T>
__device__ __forceinline__ T scan_first_order(const Grp& G, T c, const T* tab, bool asc) {
    const int NL = 32 * G.W, gl = G.gw * 32 + G.lane;
#pragma unroll
    for (int lv = 0, o = 1; o < 32; ++lv, o <<= 1) {
        const T pc = shfl_dir(c, o, asc);
        if (has_partner(G.lane, o, asc)) c = t_fma(tab[lv * NL + gl], pc, c);
    }
    return c;
}
template <typename T>
__device__ __forceinline__ void scan_second_order(const Grp& G, T& v0, T& v1, const T* tab, bool asc) {
    const int NL = 32 * G.W, gl = G.gw * 32 + G.lane;
#pragma unroll
    for (int lv = 0, o = 1; o < 32; ++lv, o <<= 1) {
        const T p0 = shfl_dir(v0, o, asc);
        const T p1 = shfl_dir(v1, o, asc);
        if (has_partner(G.lane, o, asc)) {
            const T m00 = tab[(4 * lv + 0) * NL + gl], m01 = tab[(4 * lv + 1) * NL + gl];
            const T m10 = tab[(4 * lv + 2) * NL + gl], m11 = tab[(4 * lv + 3) * NL + gl];
            const T n0 = t_fma(m00, p0, t_fma(m01, p1, v0));
            v1 = t_fma(m10, p0, t_fma(m11, p1, v1));
            v0 = n0;
        }
    }
}

// The right-hand-side part of the exclusive prefix of this lane's chunk,
// from its intra-warp inclusive value: intra-warp exclusive part, warp
// aggregates through shared memory, composition.  Two group barriers.
template <typename T>
__device__ __forceinline__ T prefix_first_order(const Grp& G, T c_incl, const T* tab, bool asc,
                                                double2* s_agg) {
    const int NL = 32 * G.W, gl = G.gw * 32 + G.lane;
    const T ex = shfl_dir(c_incl, 1, asc);
    const T c_ex = first_lane(G.lane, asc) ? t_zero(T()) : ex;
    const T agg = shfl_from(c_incl, last_lane(asc));
    if (G.lane == 0) s_agg[G.gw] = t_to2(agg);
    grp_sync(G);
    const int pw = warp_pos(G, asc);
    T P = t_zero(T());
    for (int q = 0; q < pw; ++q) {
        const int qw = asc ? q : G.W - 1 - q;
        P = t_fma(tab[7 * NL + q], P, t_from(s_agg[qw], T()));
    }
    grp_sync(G);   // the aggregates may be rewritten by the next solve
    return t_fma(tab[5 * NL + gl], P, c_ex);
}
template <typename T>
__device__ __forceinline__ void prefix_second_order(const Grp& G, T& v0, T& v1, const T* tab, bool asc,
                                                    double2* s_agg) {
    const int NL = 32 * G.W, gl = G.gw * 32 + G.lane;
    const T e0 = shfl_dir(v0, 1, asc), e1 = shfl_dir(v1, 1, asc);
    const bool first = first_lane(G.lane, asc);
    const T x0 = first ? t_zero(T()) : e0, x1 = first ? t_zero(T()) : e1;
    const int ll = last_lane(asc);
    const T a0 = shfl_from(v0, ll), a1 = shfl_from(v1, ll);
    if (G.lane == 0) { s_agg[2 * G.gw] = t_to2(a0); s_agg[2 * G.gw + 1] = t_to2(a1); }
    grp_sync(G);
    const int pw = warp_pos(G, asc);
    T p0 = t_zero(T()), p1 = t_zero(T());
    for (int q = 0; q < pw; ++q) {
        const int qw = asc ? q : G.W - 1 - q;
        const T m00 = tab[24 * NL + q], m01 = tab[25 * NL + q], m10 = tab[26 * NL + q], m11 = tab[27 * NL + q];
        const T n0 = t_fma(m00, p0, t_fma(m01, p1, t_from(s_agg[2 * qw], T())));
        p1 = t_fma(m10, p0, t_fma(m11, p1, t_from(s_agg[2 * qw + 1], T())));
        p0 = n0;
    }
    grp_sync(G);
    const T m00 = tab[20 * NL + gl], m01 = tab[21 * NL + gl], m10 = tab[22 * NL + gl], m11 = tab[23 * NL + gl];
    v0 = t_fma(m00, p0, t_fma(m01, p1, x0));
    v1 = t_fma(m10, p0, t_fma(m11, p1, x1));
}

// Output of a sweep: plain store, or out = (out + x)/2 (the H' combination).
template <typename T> __device__ __forceinline__ void put(T* out, int i, T x, bool half_add) {
    out[i] = half_add ? t_scale(t_add(out[i], x), 0.5) : x;
}

// L sweep of (LU)^{-1}: y <- L^{-1} P b (forward, with the recorded interchanges).  in != out.
// All warps of the calling group; s_agg: this group's 16-entry aggregate area.
template <typename T>
__device__ void grp_L_fwd(const Grp& G, int n, const T* __restrict__ dl, const int* __restrict__ ipiv,
                          const T* in, T* out, const T* tab, double2* s_agg) {
    const int NL = 32 * G.W, gl = G.gw * 32 + G.lane;
    const T* tb = tab + kTabL * NL;
    int lo, hi;
    grp_chunk(G, n, lo, hi);
    const int shi = min(hi, n - 1);   // steps i in [lo, shi)
    T c = t_zero(T());
    for (int i = lo; i < shi; ++i) {
        const T bn = in[i + 1];
        c = ipiv[i] == i ? t_fma(t_scale(dl[i], -1.0), c, bn) : t_fma(t_scale(dl[i], -1.0), bn, c);
    }
    c = scan_first_order(G, c, tb, true);
    c = prefix_first_order(G, c, tb, true, s_agg);
    T st = t_fma(tb[6 * NL + gl], in[0], c);
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
__device__ void grp_U_bwd(const Grp& G, int n, const T* __restrict__ e, const T* __restrict__ f,
                          const T* __restrict__ dinv, const T* y, T* out, bool half_add,
                          const T* tab, double2* s_agg) {
    const T* tb = tab + kTabU * 32 * G.W;
    int lo, hi;
    grp_chunk(G, n, lo, hi);
    T v0 = t_zero(T()), v1 = t_zero(T());
    for (int i = hi - 1; i >= lo; --i) {
        const T n0 = t_fma(e[i], v0, t_fma(f[i], v1, t_mul(y[i], dinv[i])));
        v1 = v0;
        v0 = n0;
    }
    scan_second_order(G, v0, v1, tb, false);
    prefix_second_order(G, v0, v1, tb, false, s_agg);
    T x1 = v0, x2 = v1;   // (x_{hi}, x_{hi+1})
    for (int i = hi - 1; i >= lo; --i) {
        const T x0 = t_fma(e[i], x1, t_fma(f[i], x2, t_mul(y[i], dinv[i])));
        put(out, i, x0, half_add);
        x2 = x1;
        x1 = x0;
    }
}

// U^dagger sweep: x_i = eh_i x_{i-1} + fh_i x_{i-2} + b_i conj(dinv_i) (ascending).  in != out.
template <typename T>
__device__ void grp_UH_fwd(const Grp& G, int n, const T* __restrict__ eh, const T* __restrict__ fh,
                           const T* __restrict__ dinv, const T* in, T* out,
                           const T* tab, double2* s_agg) {
    const T* tb = tab + kTabUH * 32 * G.W;
    int lo, hi;
    grp_chunk(G, n, lo, hi);
    T v0 = t_zero(T()), v1 = t_zero(T());
    for (int i = lo; i < hi; ++i) {
        const T n0 = t_fma(eh[i], v0, t_fma(fh[i], v1, t_mul(in[i], t_conj(dinv[i]))));
        v1 = v0;
        v0 = n0;
    }
    scan_second_order(G, v0, v1, tb, true);
    prefix_second_order(G, v0, v1, tb, true, s_agg);
    T x1 = v0, x2 = v1;   // (x_{lo-1}, x_{lo-2})
    for (int i = lo; i < hi; ++i) {
        const T x0 = t_fma(eh[i], x1, t_fma(fh[i], x2, t_mul(in[i], t_conj(dinv[i]))));
        out[i] = x0;
        x2 = x1;
        x1 = x0;
    }
}

// L^dagger sweep of ((LU)^dagger)^{-1} (descending, interchanges undone).  in != out.
template <typename T>
__device__ void grp_LH_bwd(const Grp& G, int n, const T* __restrict__ dl, const int* __restrict__ ipiv,
                           const T* in, T* out, bool half_add, const T* tab,
                           double2* s_agg) {
    const int NL = 32 * G.W, gl = G.gw * 32 + G.lane;
    const T* tb = tab + kTabLH * NL;
    int lo, hi;
    grp_chunk(G, n, lo, hi);
    const int shi = min(hi, n - 1);   // steps i in [lo, shi), walked downwards
    T c = t_zero(T());
    for (int i = shi - 1; i >= lo; --i)
        if (ipiv[i] == i) c = t_fma(t_scale(t_conj(dl[i]), -1.0), c, in[i]);
    c = scan_first_order(G, c, tb, false);
    c = prefix_first_order(G, c, tb, false, s_agg);
    T st = t_fma(tb[6 * NL + gl], in[n - 1], c);   // s_{shi}
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

// phase 0: p of this RHS, then steps 3-4.  With a p shared by the batch
// (Inner::p_shared) two launches: phase 1 estimates z_min, z_max of every RHS
// and stops; phase 2 takes p from the extremes over the batch and runs steps 3-4.
template <typename T>
__global__ void __launch_bounds__(256) k_inner(Inner in, int phase) {
    __shared__ double2 sh2[33];
    __shared__ double sh1[32];
    __shared__ double2 s_agg[32];   // warp aggregates of the group scans, 16 per group
    __shared__ int s_info;
    const int rhs = blockIdx.x;
    const int k = in.k, L = in.ell;
    if (in.status[rhs] != kStatusOK) {
        // no estimate from this RHS (a frozen RHS of adaptive k keeps the one
        // from the H_k it converged with)
        if (phase == 1 && threadIdx.x == 0 && in.status[rhs] != kStatusConverged) {
            in.zmin[rhs] = 0.0;
            in.zmax[rhs] = 0.0;
        }
        return;
    }
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
    T* W = reinterpret_cast<T*>(in.work + (size_t)rhs * inner_work_elems(k));
    T* tab = W + (size_t)kInnerWorkVecs * k;   // sweep tables of the current LU
    T* alT = W;                                 // H_k's diagonals as T (W[0..3k) is free)
    T* beT = W + (size_t)k;
    T* gaT = W + 2 * (size_t)k;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        alT[i] = t_from(al[i], T());
        beT[i] = t_from(be[i], T());
        gaT[i] = t_from(ga[i], T());
    }
    __syncthreads();
    T* x = W + 5 * (size_t)k;
    T* y = W + 6 * (size_t)k;
    T* vprev = W + 7 * (size_t)k;
    T* v = W + 8 * (size_t)k;
    T* r = W + 9 * (size_t)k;
    T* wprev = W + 10 * (size_t)k;
    T* w = W + 11 * (size_t)k;
    T* l = W + 12 * (size_t)k;
    const bool TS = sizeof(T) == sizeof(double2);
    const Grp G = grp_of(TS);
    double2* gagg = s_agg + 16 * G.g;

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
        sweep_tables<T>(k, dl, ipiv, e, f, eh, fh, TS, tab, s_agg);
    };

    // ---- p (Eq. popt) --------------------------------------------------------
    double p = in.p_fixed;
    if (!(p > 0.0) && phase == 2) {
        // Eq. popt with z_min = min |z| and z_max = max |z| of A, estimated as
        // the extremes over the batch's H_k (all RHS share A); every CTA forms
        // the same value in the same order
        double zmn = 0.0, zmx = 0.0;
        for (int r = 0; r < in.n_rhs; ++r) {
            const double a = in.zmin[r], b = in.zmax[r];
            if (a > 0.0 && b > 0.0 && isfinite(a) && isfinite(b)) {
                zmn = zmn > 0.0 ? fmin(zmn, a) : a;
                zmx = fmax(zmx, b);
            }
        }
        p = zmn > 0.0 ? 1.0 / sqrt(zmn * zmx) : 1.0;
    } else if (!(p > 0.0)) {
        const double x0 = 1.0 / sqrt((double)k);
        for (int i = threadIdx.x; i < k; i += blockDim.x) x[i] = t_from(mk(x0, 0.0), T());
        __syncthreads();
        double zmax = 0.0;
        for (int it = 0; it < 30; ++it) {
            band_mv<T>(k, 1.0, alT, beT, gaT, x, y, false);
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
            if (G.g == 0) {
                grp_L_fwd<T>(G, k, dl, ipiv, x, t1, tab, gagg);
                grp_sync(G);
                grp_U_bwd<T>(G, k, e, f, dinv, t1, y, false, tab, gagg);
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
                if (G.g == 0) {
                    grp_L_fwd<T>(G, k, dl, ipiv, x, t1, tab, gagg);
                    grp_sync(G);
                    grp_U_bwd<T>(G, k, e, f, dinv, t1, y, false, tab, gagg);
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
        if (phase == 1) return;
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
        band_mv<T>(k, p, alT, beT, gaT, src_r, out_r, false);
        if (TS) band_mv<T>(k, p, alT, beT, gaT, src_l, out_l, true);
        __syncthreads();
        if (G.g == 0) {
            grp_L_fwd<T>(G, k, dl, ipiv, src_r, t1, tab, gagg);
            grp_sync(G);
            grp_U_bwd<T>(G, k, e, f, dinv, t1, out_r, true, tab, gagg);
        } else if (TS) {
            grp_UH_fwd<T>(G, k, eh, fh, dinv, src_l, t2, tab, gagg);
            grp_sync(G);
            grp_LH_bwd<T>(G, k, dl, ipiv, t2, out_l, true, tab, gagg);
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
            if (!(b > 0.0)) { if (threadIdx.x == 0) in.status[rhs] = kStatusInnerBreakdown; return; }
        } else {
            double2 dlt = bdot<T>(k, r, l, sh2);        // delta <- r^dag l
            if ((dlt.x == 0.0 && dlt.y == 0.0) || !isfinite(dlt.x) || !isfinite(dlt.y)) {
                if (threadIdx.x == 0) in.status[rhs] = kStatusInnerBreakdown;
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
    T* cand_row = tmp + L;                          // [2][L] published candidate pivot row
    T* rowc = cand_row + 2 * L;                     // [2][L] published row c
    T* fcol = rowc + 2 * L;                         // [nmax]
    int* piv = reinterpret_cast<int*>(fcol + nmax); // [L]
    __shared__ double cand_val[2];
    __shared__ int cand_idx[2];
    __shared__ double part[2];
    __shared__ double sh1[32];
    __shared__ int s_stop;

    const int status0 = in.status[rhs];   // identical in every CTA of the cluster
    T* S = reinterpret_cast<T*>(in.S) + (size_t)rhs * L * L;
    const double2* alo = in.al + (size_t)rhs * L;
    const double2* blo = in.bl + (size_t)rhs * L;
    const double2* glo = in.gl + (size_t)rhs * L;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;

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
        // One cluster barrier per pivot: each CTA publishes its candidate pivot
        // row (and the owner of row c that row) in a buffer of parity c & 1
        // before the barrier; after it every CTA reads the pivot row and row c
        // from those buffers, which their owners rewrite only two pivots later,
        // after every CTA has passed the next barrier.
        for (int c = 0; c < L; ++c) {
            const int par = c & 1;
            // (a) local candidate: largest |M(i,c)|^2 over own rows i >= c (lowest i on ties);
            // nloc <= 32, so warp 0 holds one row per lane
            if (warp == 0) {
                double bv = -1.0;
                int bi = 0x7fffffff;
                if (lane < nloc) {
                    const int i = rank + C * lane;
                    if (i >= c) { bv = t_norm2(M[(size_t)lane * L + c]); bi = i; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
                }
                if (lane == 0) { cand_val[par] = bv; cand_idx[par] = bi; }
            }
            __syncthreads();
            if (cand_val[par] >= 0.0) {
                const T* src = M + (size_t)((cand_idx[par] - rank) / C) * L;
                for (int col = tid; col < L; col += blockDim.x) cand_row[par * L + col] = src[col];
            }
            if (c % C == rank) {
                const T* src = M + (size_t)(c / C) * L;
                for (int col = tid; col < L; col += blockDim.x) rowc[par * L + col] = src[col];
            }
            cl.sync();                                                  // the one barrier of the pivot
            // (b) pivot row over the cluster, ranks in fixed order (same decision everywhere)
            double pv = -1.0;
            int pi = 0x7fffffff;
            for (int q = 0; q < C; ++q) {
                double qv = cl.map_shared_rank(cand_val, q)[par];
                int qi = cl.map_shared_rank(cand_idx, q)[par];
                if (qv > pv || (qv == pv && qi < pi)) { pv = qv; pi = qi; }
            }
            if (!(pv > 0.0)) {              // singular (same decision in every CTA)
                ok = false;
                cl.sync();                  // no CTA leaves while others read its buffers
                break;
            }
            if (tid == 0) piv[c] = pi;
            // (c) fetch the pivot row and, for the owner of row pi, old row c
            {
                const T* src = cl.map_shared_rank(cand_row, pi % C) + par * L;
                for (int col = tid; col < L; col += blockDim.x) prow[col] = src[col];
                if (pi != c && pi % C == rank) {
                    const T* srcc = cl.map_shared_rank(rowc, c % C) + par * L;
                    for (int col = tid; col < L; col += blockDim.x) tmp[col] = srcc[col];
                }
            }
            __syncthreads();
            const T pinv = t_inv(prow[c]);
            // (d) multipliers of the own rows other than the pivot row, already
            // divided by the pivot (the row in slot pi now holds old row c)
            for (int li = tid; li < nloc; li += blockDim.x) {
                const int i = rank + C * li;
                const T f = (i == pi && pi != c) ? tmp[c] : M[(size_t)li * L + c];
                fcol[li] = i == c ? t_zero(T()) : t_mul(f, pinv);
            }
            __syncthreads();
            // (e) rows by warp, columns by lane: the pivot row scaled into slot c;
            // every other row: M(i,:) -= f' prow, M(i,c) = -f'
            for (int li = warp; li < nloc; li += nwarps) {
                const int i = rank + C * li;
                T* row = M + (size_t)li * L;
                if (i == c) {
                    for (int col = lane; col < L; col += 32) row[col] = col == c ? pinv : t_mul(prow[col], pinv);
                } else {
                    const T* src = (i == pi && pi != c) ? tmp : row;
                    const T f = fcol[li];
                    for (int col = lane; col < L; col += 32)
                        row[col] = col == c ? t_neg(f) : t_fma(t_neg(f), prow[col], src[col]);
                }
            }
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
    size_t smem = inner_smem_bytes(in.k, in.two_sided);   // the same for the two-float types
    const bool shared = in.p_shared && !(in.p_fixed > 0.0);
    for (int phase = shared ? 1 : 0; phase <= (shared ? 2 : 0); ++phase) {
        if (in.df_inner) {
            if (in.two_sided) k_inner<dfc><<<in.n_rhs, 256, smem, st>>>(in, phase);
            else k_inner<df><<<in.n_rhs, 256, smem, st>>>(in, phase);
        } else {
            if (in.two_sided) k_inner<double2><<<in.n_rhs, 256, smem, st>>>(in, phase);
            else k_inner<double><<<in.n_rhs, 256, smem, st>>>(in, phase);
        }
    }
}

// Largest dynamic shared memory any RHi launch needs (l <= 256, complex, 8 CTAs).
static size_t rhi_smem_max();
size_t inner_smem_bytes(int k, bool two_sided);

void init_kernel_attributes() {
    cudaFuncSetAttribute(k_inner<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)inner_smem_bytes(kMaxInnerK, false));
    cudaFuncSetAttribute(k_inner<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)inner_smem_bytes(kMaxInnerK, true));
    cudaFuncSetAttribute(k_inner<df>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)inner_smem_bytes(kMaxInnerK, false));
    cudaFuncSetAttribute(k_inner<dfc>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)inner_smem_bytes(kMaxInnerK, true));
    cudaFuncSetAttribute(k_rhi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhi_smem_max());
    cudaFuncSetAttribute(k_rhi<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rhi_smem_max());
    cudaFuncSetAttribute(k_rhi<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k_rhi<double2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    stencil32_init_attributes();
    stencil_df_init_attributes();
    lanczos_init_attributes();

}

static int rhi_cluster_size(int ell) { return ell >= 64 ? 8 : (ell >= 16 ? 4 : 1); }

template <typename T>
static size_t rhi_smem(int ell, int C) {
    int nmax = (ell + C - 1) / C;
    return (size_t)nmax * ell * sizeof(T) + 6 * (size_t)ell * sizeof(T) + (size_t)nmax * sizeof(T) +
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
    // RHi stays FP64 in every schedule: near the imaginary axis sgn is ill
    // conditioned and the iteration amplifies the working precision's rounding
    // (two-float RHi left 2 of 12 sources of the 16^3 x 32 test at 2.5e-8)
    return (int)(in.two_sided ? launch_rhi_t<double2>(in, st) : launch_rhi_t<double>(in, st));
}

void launch_inner_combine(const Inner& in, cudaStream_t st) {
    dim3 grid((in.k + 127) / 128, in.n_rhs);
    k_combine<<<grid, 128, 0, st>>>(in);
}

}  // namespace nk
