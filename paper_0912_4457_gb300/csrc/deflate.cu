// LR deflation of the critical eigenpairs (App. C steps 1 and 6) on vectors
// in the ABI layout, batched over the RHS:
//   step 1:  d_{r,i} = <l_i, b_r>,  x_minus_r = b_r - sum_i d_{r,i} r_i,
//   step 6:  y_r += sum_i sgn(lambda_i) d_{r,i} r_i   (sgn(z) = sgn(Re z), Eq. sgnz),
// with <l_i, r_j> = delta_ij (l_i = r_i for Hermitian A).  All arithmetic is
// FP64; the dot products use a fixed summation order (one block per
// eigenvector and RHS), so a solve is bitwise reproducible.
#include "nk_common.cuh"
#include "nk_kernels.h"

namespace nk {

namespace {

constexpr int kThreads = 256;

// d[r * m + i] = sum_n conj(L_i[n]) b_r[n]
__global__ void __launch_bounds__(kThreads) k_defl_dots(const double2* __restrict__ L, const double2* __restrict__ b,
                                                        long N, int m, double2* __restrict__ d) {
    __shared__ double2 sh[33];
    const int i = blockIdx.x, r = blockIdx.y;
    const double2* li = L + (size_t)i * N;
    const double2* br = b + (size_t)r * N;
    double2 acc = mk(0.0, 0.0);
    for (long n = threadIdx.x; n < N; n += blockDim.x) {
        const double2 l = li[n], x = br[n];
        acc.x = fma(l.x, x.x, fma(l.y, x.y, acc.x));   // conj(l) x
        acc.y = fma(l.x, x.y, fma(-l.y, x.x, acc.y));
    }
    const double2 t = block_sum(acc, sh);
    if (threadIdx.x == 0) d[(size_t)r * m + i] = t;
}

// out_r[n] = base_r[n] + sum_i w_i d[r * m + i] R_i[n], with w_i = -1 (step 1)
// or sgn(Re lambda_i) (step 6, sgn given in w); out may alias base.
__global__ void __launch_bounds__(kThreads) k_defl_axpy(const double2* base, double2* out,
                                                        const double2* __restrict__ R, const double2* __restrict__ d,
                                                        const double* __restrict__ w, long N, int m) {
    extern __shared__ double2 coef[];   // [m]: w_i d_{r,i} of this RHS
    const int r = blockIdx.y;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double2 v = d[(size_t)r * m + i];
        coef[i] = mk(w[i] * v.x, w[i] * v.y);
    }
    __syncthreads();
    const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double2 acc = base[(size_t)r * N + n];
    for (int i = 0; i < m; ++i) {
        const double2 c = coef[i], v = R[(size_t)i * N + n];
        acc.x = fma(c.x, v.x, fma(-c.y, v.y, acc.x));
        acc.y = fma(c.x, v.y, fma(c.y, v.x, acc.y));
    }
    out[(size_t)r * N + n] = acc;
}

// y_r = b_r + gamma5 y_r (ABI layout: component 12 site + 3 spin + colour;
// gamma5 = diag(1, 1, -1, -1) in spin)
__global__ void k_overlap_finish(const double2* __restrict__ b, double2* y, long N, int n) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)N * n) return;
    const int c = (int)(t % 12);
    const double g = c < 6 ? 1.0 : -1.0;
    const double2 v = y[t], x = b[t];
    y[t] = mk(x.x + g * v.x, x.y + g * v.y);
}

}  // namespace

void launch_defl_dots(const double2* L, const double2* b, long N, int m, int n_rhs, double2* d, cudaStream_t st) {
    k_defl_dots<<<dim3(m, n_rhs), kThreads, 0, st>>>(L, b, N, m, d);
}

void launch_defl_axpy(const double2* base, double2* out, const double2* R, const double2* d, const double* w, long N,
                      int m, int n_rhs, cudaStream_t st) {
    const dim3 grid((unsigned)((N + kThreads - 1) / kThreads), n_rhs);
    k_defl_axpy<<<grid, kThreads, sizeof(double2) * (size_t)m, st>>>(base, out, R, d, w, N, m);
}

void launch_overlap_finish(const double2* b, double2* y, long N, int n, cudaStream_t st) {
    const size_t tot = (size_t)N * n;
    k_overlap_finish<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(b, y, N, n);
}

}  // namespace nk
