// Device part of the eigensolver of the deflation (nk_eigs_smallest,
// engine.cu): Ritz vectors as combinations of the stored basis columns,
//   out_i = sum_j coef[i][j] base_j,
// FP64 with explicit FMA chains (the Ritz vectors of App. A / B's bases
// V_k and W_k, coefficients from the eigenvectors of H_k).
#include "nk_common.cuh"
#include "nk_kernels.h"

namespace nk {

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_colcomb(const double2* __restrict__ base, long col_stride, int ncols,
                                                     const double2* __restrict__ coef, long N,
                                                     double2* __restrict__ out) {
    const int i = blockIdx.y;
    const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double2* c = coef + (size_t)i * ncols;
    double2 acc = mk(0.0, 0.0);
    for (int j = 0; j < ncols; ++j) {
        const double2 cj = __ldg(c + j), v = __ldg(base + (size_t)j * col_stride + n);
        acc.x = fma(cj.x, v.x, fma(-cj.y, v.y, acc.x));
        acc.y = fma(cj.x, v.y, fma(cj.y, v.x, acc.y));
    }
    out[(size_t)i * N + n] = acc;
}

}  // namespace

void launch_colcomb(const double2* base, long col_stride, int ncols, const double2* coef, long N, int n_out,
                    double2* out, cudaStream_t st) {
    const dim3 grid((unsigned)((N + kThreads - 1) / kThreads), (unsigned)n_out);
    k_colcomb<<<grid, kThreads, 0, st>>>(base, col_stride, ncols, coef, N, out);
}

}  // namespace nk
