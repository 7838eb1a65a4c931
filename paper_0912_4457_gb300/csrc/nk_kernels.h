// Internal kernel interfaces shared by the .cu files of the library (not part
// of the C ABI; see include/nksign.h for that).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nk {

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
void launch_links_to_device_layout(const double2* in, double2* u64, float2* u32, int V,
                                   cudaStream_t st);
void launch_abi_to_soa(const double2* in, long in_stride, double2* out, long out_stride, int V,
                       int n, cudaStream_t st);
void launch_soa_to_abi(const double2* in, long in_stride, double2* out, long out_stride,
                       const double2* add, long add_stride, int V, int n, cudaStream_t st);
void launch_to_fp32(const double2* in, long in_stride, float2* out, long out_stride, long N, int n,
                    cudaStream_t st);

// ---- outer (two-sided) Lanczos recurrence -------------------------------------

// Device buffers of one batched outer recurrence; all per-RHS arrays are
// indexed [rhs][...].
struct Outer {
    long N;          // vector length (12 V complex)
    int n_rhs, k, nblk;
    int two_sided;
    double2* V;      // basis, [rhs][k][N] (single pass) -- or nullptr
    double2* vring;  // [rhs][2][N] ring of v_{j-1}, v_j when V == nullptr (double pass)
    double2* w;      // [rhs][2][N] ring of w_{j-1}, w_j (two-sided)
    double2* r;      // [rhs][N]
    double2* l;      // [rhs][N]
    double2* s;      // stencil output A v_j, [rhs][N]
    double2* t;      // stencil output A^dagger w_j, [rhs][N]
    float2* v32;     // FP32 copy of v_j, [rhs][N]
    float2* w32;     // FP32 copy of w_j, [rhs][N]
    double2* alpha;  // H(j,j), [rhs][k]
    double2* beta;   // H(j+1,j), [rhs][k]
    double2* gamma;  // H(j,j+1), [rhs][k]
    double2* partials;  // [rhs][nblk]
    unsigned* counters; // [rhs]
    int* status;        // [rhs]
    double* xnorm;      // [rhs]
    double2* y;         // double-pass accumulation y = sum_j c_j v_j, [rhs][N]
    const double2* c;   // double-pass coefficients, [rhs][k]
};

__host__ __device__ inline double2* outer_v(const Outer& o, int rhs, int j) {
    return o.V ? o.V + ((size_t)rhs * o.k + j) * o.N : o.vring + ((size_t)rhs * 2 + (j & 1)) * o.N;
}
__host__ __device__ inline double2* outer_w(const Outer& o, int rhs, int j) {
    return o.w + ((size_t)rhs * 2 + (j & 1)) * o.N;
}

// status codes kept on the device (0 = fine)
constexpr int kStatusOK = 0;
constexpr int kStatusZeroSource = 1;  // |b| = 0: result is 0
constexpr int kStatusBreakdown = 2;   // two-sided serious breakdown
constexpr int kStatusRhi = 3;         // RHi did not converge / singular pivot
constexpr int kStatusLU = 4;          // singular p H_k

void launch_outer_init(const Outer& o, const double2* b_soa, int write32, cudaStream_t st);
void launch_outer_step1(const Outer& o, int j, cudaStream_t st);
void launch_outer_step2(const Outer& o, int j, cudaStream_t st);
void launch_outer_step3(const Outer& o, int j, int write32, cudaStream_t st);
void launch_lift(const Outer& o, const double2* c, double2* y, cudaStream_t st);

// ---- inner part: p estimate, LU of p H_k, inner Lanczos, RHi, c = V_l s -------

struct Inner {
    int n_rhs, k, ell;
    int two_sided;
    const double2* alpha;  // outer H_k, [rhs][k]
    const double2* beta;
    const double2* gamma;
    double p_fixed;        // > 0: use it; else estimate
    double* p;             // [rhs] out
    double* zmin;          // [rhs] out
    double* zmax;          // [rhs] out
    double2* work;         // [rhs][kInnerWorkVecs][k] scratch
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
    int* timeout;          // device flag: a bounded wait ran out
};
constexpr int kInnerWorkVecs = 16;

void launch_inner_lanczos(const Inner& in, cudaStream_t st);
int launch_rhi(const Inner& in, cudaStream_t st);  // returns cudaError_t
void launch_inner_combine(const Inner& in, cudaStream_t st);
// Kernel attributes that must be set outside stream capture (once per device).
void init_kernel_attributes();

}  // namespace nk
