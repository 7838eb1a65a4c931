// Vector kernels of the overlap inversion (nk_overlap_solve): conjugate
// gradients on the normal equations of M = D_ov(mu) + m, each iteration
// applying M and M^dagger through the nested sign function.  Vectors are in
// the ABI layout (12 V complex per RHS), batched over n RHS with one scalar
// per RHS; FP64 throughout, dot products in a fixed summation order.
#include "nk_common.cuh"
#include "nk_kernels.h"

namespace nk {

namespace {

constexpr int kThreads = 256;

// out[r] = sum_n conj(a_r[n]) b_r[n], one block per RHS
__global__ void __launch_bounds__(kThreads) k_vdot(const double2* __restrict__ a, const double2* __restrict__ b,
                                                   long N, double2* __restrict__ out) {
    __shared__ double2 sh[33];
    const size_t base = (size_t)blockIdx.x * N;
    double2 acc = mk(0.0, 0.0);
    for (long n = threadIdx.x; n < N; n += blockDim.x) {
        const double2 x = a[base + n], y = b[base + n];
        acc.x = fma(x.x, y.x, fma(x.y, y.y, acc.x));
        acc.y = fma(x.x, y.y, fma(-x.y, y.x, acc.y));
    }
    const double2 t = block_sum(acc, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
}

// y_r = ca_r x_r + cb_r y_r (complex per-RHS coefficients)
__global__ void k_vlincomb(double2* y, const double2* __restrict__ x, long N, VecCoefs ca, VecCoefs cb) {
    const int r = blockIdx.y;
    const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const size_t i = (size_t)r * N + n;
    const double2 a = ca.c[r], b = cb.c[r], u = x[i], v = y[i];
    y[i] = mk(fma(a.x, u.x, fma(-a.y, u.y, fma(b.x, v.x, -b.y * v.y))),
              fma(a.x, u.y, fma(a.y, u.x, fma(b.x, v.y, b.y * v.x))));
}

// v_r <- gamma5 v_r (ABI layout: gamma5 = diag(1, 1, -1, -1) in spin)
__global__ void k_gamma5(double2* v, long N, int n) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)N * n) return;
    if (t % 12 >= 6) v[t] = mk(-v[t].x, -v[t].y);
}

}  // namespace

void launch_vdot(const double2* a, const double2* b, long N, int n, double2* out, cudaStream_t st) {
    k_vdot<<<n, kThreads, 0, st>>>(a, b, N, out);
}

void launch_vlincomb(double2* y, const double2* x, long N, int n, const VecCoefs& ca, const VecCoefs& cb,
                     cudaStream_t st) {
    const dim3 grid((unsigned)((N + kThreads - 1) / kThreads), n);
    k_vlincomb<<<grid, kThreads, 0, st>>>(y, x, N, ca, cb);
}

void launch_gamma5(double2* v, long N, int n, cudaStream_t st) {
    const size_t tot = (size_t)N * n;
    k_gamma5<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(v, N, n);
}

}  // namespace nk
