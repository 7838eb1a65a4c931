// Internal kernel interfaces shared by the .cu files of the library (not part
// of the C ABI; see include/nksign.h for that).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nk {

struct dfc;   // two-float complex (nk_common.cuh)

struct Geom {
    int Lx, Ly, Lz, Lt, V;
    int antiperiodic;
};

// A set of vectors for one stencil launch: out_i = A in_i (dag = 0) or A^dagger in_i.
// `in` is double2* for the FP64 stencil and float2* for the FP32 one.
struct DslashSet {
    const void* in;
    long in_stride;   // elements (complex) between consecutive vectors
    double2* out;
    long out_stride;
    int n;
    int dag;
};

void launch_dslash(int precision, const void* U, const Geom& g, const DslashSet& s0,
                   const DslashSet& s1, double kappa, double mu, cudaStream_t st);
void launch_links_to_device_layout(const double2* in, double2* u64, float2* u32, dfc* udf, int V,
                                   cudaStream_t st);
int plaquette_blocks(const Geom& g);
void launch_plaquette(const double2* U, const Geom& g, double* partial, cudaStream_t st);
void launch_to_df(const double2* in, long in_stride, dfc* out, long out_stride, long N, int n, cudaStream_t st);
void launch_abi_to_soa(const double2* in, long in_stride, double2* out, long out_stride, int V,
                       int n, cudaStream_t st);
void launch_soa_to_abi(const double2* in, long in_stride, double2* out, long out_stride,
                       const double2* add, long add_stride, int V, int n, cudaStream_t st);
// ABI spinors (double, [site][12]) <-> FP32 pair layout ([6][V] float4), n vectors
void launch_abi_to_f32pair(const double2* in, long in_stride, float4* out, long out_stride, int V, int n,
                           cudaStream_t st);
void launch_f32pair_to_abi(const float4* in, long in_stride, double2* out, long out_stride, int V, int n,
                           cudaStream_t st);

// The multi-RHS FP32 stencil alone (stencil32.cu): out = A in for the n_a
// vectors of in_a, A^dagger in for the n_d vectors of in_d; FP32 pair layout,
// vstride float4 between vectors; n_a + n_d <= 24.  With scale set (the
// step scalars of an outer recurrence, [rhs][kScalars]) output vector i of
// A is multiplied by scale[i][kScN] (1/n_j) and of A^dagger by
// scale[i][kScM] (1/m_j), in FP32: the application A v_j, A^dagger w_j of
// the unnormalised basis.
struct Stencil32Set {
    const float4* in_a;
    const float4* in_d;
    float4* out_a;
    float4* out_d;
    long vstride;
    int n_a, n_d;
    const double2* scale;
};
void launch_stencil32(const void* U32, const Geom& g, const Stencil32Set& s, double kappa, double mu,
                      cudaStream_t st);

// The multi-RHS two-float stencil (stencil_df.cu): out = A in for the n_a
// vectors of in_a, A^dagger in for the n_d vectors of in_d; two-float input
// and FP64 output vectors in the layout [12][V], in_stride / out_stride
// elements between vectors; n_a + n_d <= 24.  With scale set (the step
// scalars, [rhs][kScalars]) output vector i of A is multiplied by
// scale[i][kScN] and of A^dagger by scale[i][kScM] in two-float arithmetic.
struct StencilDfSet {
    const dfc* in_a;
    const dfc* in_d;
    double2* out_a;
    double2* out_d;
    long in_stride, out_stride;
    int n_a, n_d;
    const double2* scale;
};
void launch_stencil_df(const void* Udf, const Geom& g, const StencilDfSet& s, double kappa, double mu,
                       cudaStream_t st);
void stencil_df_init_attributes();   // dynamic shared memory (outside capture)
int stencil32_sites_per_cta(int nv);
void stencil32_init_attributes();   // dynamic shared memory above 48 KB (outside capture)
int stencil32_blocks(const Geom& g, int nv);

// ---- outer (two-sided) Lanczos recurrence -------------------------------------

// Device buffers of one batched outer recurrence; per-RHS arrays are indexed
// [rhs][...].  Basis vectors are stored unnormalised (see lanczos.cu):
// q_j = n_j v_j and p_j = m_j w_j.
struct Outer {
    long N;          // vector length (12 V complex)
    int n_rhs, k, nblk, npart;
    int st_threads;  // fused stencil: sites (threads) per CTA, 64 / 128 / 256
    int st_order;    // fused stencil grid: 0 vector-fastest (link reuse in L2), 1 site-block-fastest
    int st_split;    // fused stencil: threads per site, 1 or 3 (one colour each)
    int st_threads_df, st_order_df, st_split_df;   // the same for the two-float stencil steps
    int two_sided;
    int q_ring;      // 0: Q holds all k vectors (+1 scratch) [rhs][k+1][N]; 1: ring [rhs][3][N] (double pass)
    int qcols;       // vectors per RHS in Q: k + 1 or 3
    double2* Q;      // right basis q_j
    double2* P;      // left vectors p_j, ring [rhs][3][N] (two-sided), or all [rhs][k+1][N] (pcols = k + 1)
    int pcols;       // vectors per RHS in P: 3 (ring) or k + 1 (the eigensolver keeps W_k)
    float4* q32;     // FP32 copy of the newest q, [rhs][6][V] pair layout (f32_pair_index)
    float4* p32;     // FP32 copy of the newest p, [rhs][6][V]
    float4* s32;     // FP32 stencil output of the step, (A q_j)/n_j then (A^dag p_j)/m_j: [side][rhs][6][V]
    double2* s64;    // the same from the two-float stencil, FP64: [side][rhs][12][V]
    dfc* qdf;        // two-float copy of the newest q, [rhs][N]
    dfc* pdf;        // two-float copy of the newest p, [rhs][N]
    double2* alpha;  // H(j,j), [rhs][k]
    double2* beta;   // H(j+1,j), [rhs][k]
    double2* gamma;  // H(j,j+1), [rhs][k]
    double2* partials;  // [rhs][npart]
    unsigned* counters; // [rhs]; the all-RHS kernels (k_stencil32_step1) use counters[0]
    double2* sc;        // [rhs][kScalars]: scalars of the current outer step (below)
    int* status;        // [rhs]
    double* xnorm;      // [rhs]
    double2* y;         // double pass: accumulation y = sum_j c'_j q_j, [rhs][N]
    const double2* cp;  // double pass: lift coefficients c'_j, [rhs][k]
    // Mixed schedule (NK_MIXED): two-float rings of the newest three right and
    // left vectors, [rhs][3][N] (slot j % 3).  The early (two-float stencil)
    // steps run in FP64 and copy their new vectors into the rings, which the
    // two-float stencil reads; the late (FP32 stencil) steps run in two-float
    // arithmetic from the rings, keeping only the right basis also in FP64
    // (Q, for the lift).  nullptr in the all-FP64 schedule.
    dfc* qr;
    dfc* pr;
    // Q columns from q_df_from on hold two-float values (dfc, 16 bytes like
    // double2): the late steps of the mixed schedule, whose recurrence runs in
    // two-float arithmetic, write them without an FP64 conversion, and the
    // two-float lift reads them as they are.  Larger than k otherwise.
    int q_df_from;
    // Mixed schedule: steps j >= ring_from run the recurrence (the stencil
    // kernel's epilogue and step 2) in two-float arithmetic on the rings;
    // the steps before it in FP64.  Larger than k (the default): the whole
    // recurrence in FP64.
    int ring_from;
};

__host__ __device__ inline double2* outer_q(const Outer& o, int rhs, int j) {
    return o.Q + ((size_t)rhs * o.qcols + (o.q_ring ? j % 3 : j)) * o.N;
}
__host__ __device__ inline double2* outer_p(const Outer& o, int rhs, int j) {
    return o.P + ((size_t)rhs * o.pcols + (o.pcols == 3 ? j % 3 : j)) * o.N;
}
// (byte arithmetic: dfc, a two-float complex of 16 bytes, may be incomplete here)
__host__ __device__ inline dfc* ring_q(const Outer& o, int rhs, int j) {
    return reinterpret_cast<dfc*>(reinterpret_cast<char*>(o.qr) + ((size_t)rhs * 3 + j % 3) * o.N * 16);
}
__host__ __device__ inline dfc* ring_p(const Outer& o, int rhs, int j) {
    return reinterpret_cast<dfc*>(reinterpret_cast<char*>(o.pr) + ((size_t)rhs * 3 + j % 3) * o.N * 16);
}
// n_j (q_j = n_j v_j) and m_j (p_j = m_j w_j)
__device__ inline double2 scale_n(const Outer& o, int rhs, int j) {
    return j == 0 ? make_double2(o.xnorm[rhs], 0.0) : o.beta[(size_t)rhs * o.k + j - 1];
}
__device__ inline double2 scale_m(const Outer& o, int rhs, int j) {
    if (j == 0) return make_double2(o.xnorm[rhs], 0.0);
    double2 g = o.gamma[(size_t)rhs * o.k + j - 1];
    return make_double2(g.x, -g.y);
}

// Scalars of outer step j per RHS (complex FP64), formed once per step by the
// finishing block of the kernel that completes their inputs -- the norm kernel
// (j = 0) or step 2 of step j - 1 (kScN .. kScC1L), the step-1 kernel (kScC3,
// kScC4) -- so that the kernels of the step read them instead of each CTA
// dividing again (FP64 divisions are slow on GB300).
constexpr int kScalars = 8;
constexpr int kScN = 0;    // 1/n_j: scale of the stencil output A q_j
constexpr int kScC1 = 1;   // c_{j-1}/n_{j-1} (c = gamma two-sided, beta Hermitian); 0 at j = 0
constexpr int kScD = 2;    // 1/m_j^* two-sided, 1/n_j Hermitian: H(j,j) = kScD x (dot of r)
constexpr int kScM = 3;    // 1/m_j: scale of A^dagger p_j
constexpr int kScC1L = 4;  // beta_{j-1}^*/m_{j-1}; 0 at j = 0
constexpr int kScC3 = 5;   // H(j,j)/n_j (step 2, right)
constexpr int kScC4 = 6;   // H(j,j)^*/m_j (step 2, left)

// FP32 vectors are stored in the pair layout [6][V] of float4 per vector:
// float4 i of site s holds spin-colour components 2i and 2i + 1.  As float2
// elements (one complex each), component c of site s is element:
__host__ __device__ inline size_t f32_pair_index(int c, int s, int V) {
    return 2 * ((size_t)(c >> 1) * V + s) + (c & 1);
}

// status codes kept on the device (0 = fine)
constexpr int kStatusOK = 0;
constexpr int kStatusZeroSource = 1;  // |b| = 0: result is 0
constexpr int kStatusBreakdown = 2;   // serious breakdown (or a zero beta)
constexpr int kStatusRhi = 3;         // RHi did not converge / singular pivot
constexpr int kStatusLU = 4;          // singular p H_k
constexpr int kStatusConverged = 5;   // adaptive k: frozen at its converged size (skipped by the kernels)
constexpr int kStatusInnerBreakdown = 6;  // inner (two-sided) Lanczos on H_k': zero beta or delta
constexpr int kStatusTimeout = 7;     // a bounded wait of a streaming kernel ran out (copies never landed)

// First failure of an RHS wins (a later one does not overwrite it).
__device__ inline void mark_failed(const Outer& o, int rhs, int code) { atomicCAS(o.status + rhs, kStatusOK, code); }

// Copy modes for the next stencil's input: none, FP32, two-float.
constexpr int kCopyNone = 0, kCopy32 = 1, kCopyDF = 2;
// keep_status: the second pass of NK_DOUBLE_PASS (a failure of the first pass stays)
void launch_outer_init(const Outer& o, int copy_mode, cudaStream_t st, bool keep_status = false);
// Stencil + first half of step j; precision 32 (FP32, the multi-RHS stencil
// of stencil32.cu, then the FP64 step-1 kernel of lanczos.cu; fused with a
// two-float epilogue in the two-float recurrence), 48 (two-float) or 64
// (FP64) (dslash.cu).  Returns the number of kernels launched.
int launch_dslash_step1(int precision, const void* U, const Geom& g, const Outer& o, int j,
                        double kappa, double mu, cudaStream_t st);
// The FP32 and two-float steps of an FP64 recurrence (precision 32 or 48
// before o.ring_from, with o.s32 / o.s64): the multi-RHS stencil, which leaves
// s = (A q_j)/n_j and t = (A^dag p_j)/m_j in o.s32 (FP32) or o.s64 (FP64 from
// the two-float stencil) (dslash.cu), then the first half of outer step j in
// FP64 (lanczos.cu).
bool split_step(int precision, const Outer& o, int j);
void launch_stencil_step(int precision, const void* U, const Geom& g, const Outer& o, int j, double kappa,
                         double mu, cudaStream_t st);
void launch_outer_step1(const Outer& o, int j, bool s64, cudaStream_t st);
void lanczos_init_attributes();   // dynamic shared memory above 48 KB (outside capture)
int stream_ctas_per_sm();         // CTAs of the streaming step kernels per SM
int stream_tile_sites();          // sites per tile of the streaming step kernels
void launch_stencil32_step1(const void* U32, const Geom& g, const Outer& o, int j, double kappa, double mu,
                            cudaStream_t st);
int dslash_step1_blocks(const Geom& g, int threads);
constexpr int kStencilMaxThreads = 256;
// ring: the step belongs to the two-float recurrence of the mixed schedule
// (j >= ring_from), which runs on the two-float rings; otherwise FP64, and
// write_ring says whether the FP64 step also stores two-float copies of its
// new vectors in the rings (for a two-float stencil or a later ring step).
void launch_outer_step2(const Outer& o, int j, int copy_mode, bool ring, bool write_ring, cudaStream_t st);
// kused[rhs]: outer steps whose basis vectors enter the lift of that RHS (k or,
// adaptive, the converged size); coefficients beyond it are zero.
void launch_lift_coef(const Outer& o, const double2* c, const int* kused, double2* cp, cudaStream_t st);
void launch_lift(const Outer& o, const double2* cp, const int* kused, double2* y, cudaStream_t st);
// out_i = sum_{j < ncols} coef[i ncols + j] base[j col_stride + n] for the n_out
// output vectors i (eigen.cu): Ritz vectors from a stored basis
void launch_colcomb(const double2* base, long col_stride, int ncols, const double2* coef, long N, int n_out,
                    double2* out, cudaStream_t st);
void launch_fill_int(int* p, int n, int value, cudaStream_t st);
// Adaptive k: per RHS (|c - c_prev|, |c|) over the first k entries, then c_prev <- c.
void launch_adapt_delta(const Outer& o, const double2* c, double2* c_prev, int k, double2* dn, cudaStream_t st);
// LR deflation (deflate.cu), ABI-layout vectors of N complex: d[r m + i] = <l_i, b_r>;
// out_r = base_r + sum_i w_i d[r m + i] R_i (out may alias base); y_r = b_r + gamma5 y_r
void launch_defl_dots(const double2* L, const double2* b, long N, int m, int n_rhs, double2* d, cudaStream_t st);
void launch_defl_axpy(const double2* base, double2* out, const double2* R, const double2* d, const double* w, long N,
                      int m, int n_rhs, cudaStream_t st);
void launch_overlap_finish(const double2* b, double2* y, long N, int n, cudaStream_t st);
// Overlap inversion (overlap.cu), ABI-layout vectors, n <= 12 RHS:
// out[r] = <a_r, b_r>; y_r = ca_r x_r + cb_r y_r; v_r <- gamma5 v_r
struct VecCoefs {
    double2 c[12];
};
void launch_vdot(const double2* a, const double2* b, long N, int n, double2* out, cudaStream_t st);
void launch_vlincomb(double2* y, const double2* x, long N, int n, const VecCoefs& ca, const VecCoefs& cb,
                     cudaStream_t st);
void launch_gamma5(double2* v, long N, int n, cudaStream_t st);
// NK_EPS_EST: per RHS (|x2 - b|^2, |b|^2) of n vectors of N complex (any common layout)
void launch_eps_sums(const double2* b, const double2* x2, int n, long N, double2* out, cudaStream_t st);

// ---- inner part: p estimate, LU of p H_k, inner Lanczos, RHi, c = V_l s -------

struct Inner {
    int n_rhs, k, ell;
    int kstride;           // row stride of alpha/beta/gamma and c (0: k); the adaptive
                           // mode runs the inner part on the leading k x k block of H
    int two_sided;
    const double2* alpha;  // outer H_k, [rhs][k]
    const double2* beta;
    const double2* gamma;
    double p_fixed;        // > 0: use it; else estimate
    int p_shared;          // 1: one p for the batch, from the extremes of the z_min, z_max
                           // estimates over its RHS (all RHS share A); 0: p per RHS
    double* p;             // [rhs] out
    double* zmin;          // [rhs] out
    double* zmax;          // [rhs] out
    double2* work;         // [rhs][inner_work_elems(k)] scratch
    int* ipiv;             // [rhs][k]
    double2* Vl;           // inner basis [rhs][ell][k]
    double2* al;           // inner H_l, [rhs][ell]
    double2* bl;
    double2* gl;
    double2* S;            // RHi iterate, [rhs][ell][ell]
    double2* s;            // sgn(H_l) e_1, [rhs][ell]
    int* rhi_iters;        // [rhs]
    double2* c;            // V_l s, [rhs][k]
    int* status;           // [rhs]
    int df_inner;          // 1: p estimate, LU, sweeps and inner Lanczos in two-float
                           // arithmetic (the mixed schedule); 0: FP64
};
constexpr int kInnerWorkVecs = 16;
// per RHS: kInnerWorkVecs vectors of length k, then the sweep tables of the LU
constexpr int kSweepTableElems = 72 * 256;   // 72 table rows x up to 256 group lanes
__host__ __device__ constexpr size_t inner_work_elems(int k) { return (size_t)kInnerWorkVecs * k + kSweepTableElems; }
// Largest outer size k the inner kernel supports (its LU factors and solve
// vectors, 8 complex vectors of length k plus the pivots, fill shared memory).
constexpr int kMaxInnerK = 1536;

void launch_inner_lanczos(const Inner& in, cudaStream_t st);
// kernels launch_inner_lanczos launches: two with a p shared by the batch
inline int inner_launches(const Inner& in) { return in.p_shared && !(in.p_fixed > 0.0) ? 2 : 1; }
int launch_rhi(const Inner& in, cudaStream_t st);  // returns cudaError_t
void launch_inner_combine(const Inner& in, cudaStream_t st);
// Kernel attributes that must be set outside stream capture (once per device).
void init_kernel_attributes();

}  // namespace nk
