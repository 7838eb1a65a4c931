// nk_inner_sign_noalloc: the inner half of the nested method (p estimate,
// LU of p H_k, inner Lanczos with H_k', Roberts-Higham on H_l, c = V_l s)
// for callers that cannot allocate device memory -- code that runs where
// cudaMalloc is forbidden or unsafe (inside another framework's memory
// budget, in a process whose allocator is owned by someone else, or on a
// real-time path that must not allocate).  Its scratch lives in the
// file-scope device array below instead of memory the context would
// allocate; the caller passes only its inputs and outputs.
//
// The array is a module global: every GPU that loads this library holds it
// (about 5.9 MB) until the process exits.  All calls share it and it keeps the
// last call's contents, so calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it; serialise them.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "../../include/nksign.h"
#include "nk_kernels.h"

namespace {

constexpr int kMaxRhs = NK_NOALLOC_MAX_RHS;
constexpr int kMaxK = NK_NOALLOC_MAX_K;
constexpr int kMaxEll = NK_NOALLOC_MAX_ELL;

// Scratch layout, in units of double2 (16 bytes), each piece 256-byte aligned.
constexpr size_t kAlign = 16;  // 16 double2 = 256 bytes
constexpr size_t up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffWork = 0;
constexpr size_t kOffVl = kOffWork + up((size_t)kMaxRhs * nk::inner_work_elems(kMaxK));
constexpr size_t kOffS = kOffVl + up((size_t)kMaxRhs * kMaxEll * kMaxK);
constexpr size_t kOffAl = kOffS + up((size_t)kMaxRhs * kMaxEll * kMaxEll);
constexpr size_t kOffBl = kOffAl + up((size_t)kMaxRhs * kMaxEll);
constexpr size_t kOffGl = kOffBl + up((size_t)kMaxRhs * kMaxEll);
constexpr size_t kOffSv = kOffGl + up((size_t)kMaxRhs * kMaxEll);
constexpr size_t kOffP = kOffSv + up((size_t)kMaxRhs * kMaxEll);       // p, z_min, z_max (doubles)
constexpr size_t kOffInt = kOffP + up((size_t)3 * kMaxRhs);            // ipiv, status, iters (ints)
constexpr size_t kInts = (size_t)kMaxRhs * kMaxK + 2 * kMaxRhs;
constexpr size_t kTotal = kOffInt + up((kInts + 3) / 4);

__device__ __align__(256) double2 g_noalloc_scratch[kTotal];

// Device address of the array, looked up once per device (host code must not
// use the symbol itself: on the host it only stands in for the device array).
double2* g_scratch_addr[64] = {nullptr};

int set_err(char* err, size_t n, int code, const char* msg) {
    if (err && n) {
        std::strncpy(err, msg, n - 1);
        err[n - 1] = '\0';
    }
    return code;
}

}  // namespace

extern "C" int nk_inner_sign_noalloc(const double* alpha_dev, const double* beta_dev, const double* gamma_dev,
                                     int n_rhs, int k, int ell, double p, int hermitian, double* c_dev,
                                     void* stream, char* err, size_t err_len) {
    if (!alpha_dev || !beta_dev || !gamma_dev || !c_dev)
        return set_err(err, err_len, NK_EINVAL, "null pointer");
    if (n_rhs < 1 || k < 2 || ell < 2 || ell > k || (k & 1) || (ell & 1))
        return set_err(err, err_len, NK_EINVAL, "need n_rhs >= 1 and even 2 <= l <= k");
    if (n_rhs > kMaxRhs || k > kMaxK || ell > kMaxEll) {
        char msg[160];
        std::snprintf(msg, sizeof(msg),
                      "size beyond the static scratch: need n_rhs <= %d, k <= %d, l <= %d (got %d, %d, %d)",
                      kMaxRhs, kMaxK, kMaxEll, n_rhs, k, ell);
        return set_err(err, err_len, NK_EINVAL, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64)
        return set_err(err, err_len, NK_ECUDA, "cudaGetDevice failed");
    if (!g_scratch_addr[dev]) {
        // first call on this device: resolve the array's device address and
        // set the kernel attributes the RHi launch needs
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return set_err(err, err_len, NK_ECUDA, cudaGetErrorString(e));
        nk::init_kernel_attributes();
        cudaGetLastError();
        g_scratch_addr[dev] = (double2*)ptr;
    }
    double2* base = g_scratch_addr[dev];
    cudaStream_t st = (cudaStream_t)stream;
    nk::Inner in;
    std::memset(&in, 0, sizeof(in));
    in.n_rhs = n_rhs;
    in.k = k;
    in.ell = ell;
    in.two_sided = hermitian ? 0 : 1;
    in.alpha = (const double2*)alpha_dev;
    in.beta = (const double2*)beta_dev;
    in.gamma = (const double2*)gamma_dev;
    // p > 0 fixes p; p == 0 estimates one p per RHS; p < 0 one p for the
    // batch, from the extremes of the per-RHS estimates (as nk_inner_sign)
    in.p_fixed = p > 0.0 ? p : 0.0;
    in.p_shared = p < 0.0 ? 1 : 0;
    in.work = base + kOffWork;
    in.Vl = base + kOffVl;
    in.S = base + kOffS;
    in.al = base + kOffAl;
    in.bl = base + kOffBl;
    in.gl = base + kOffGl;
    in.s = base + kOffSv;
    double* dbl = (double*)(base + kOffP);
    in.p = dbl;
    in.zmin = dbl + kMaxRhs;
    in.zmax = dbl + 2 * kMaxRhs;
    int* ints = (int*)(base + kOffInt);
    in.ipiv = ints;
    in.status = ints + (size_t)kMaxRhs * kMaxK;
    in.rhi_iters = in.status + kMaxRhs;
    in.c = (double2*)c_dev;
    // the array keeps the previous call's contents: the status flags must start at 0
    e = cudaMemsetAsync(in.status, 0, sizeof(int) * n_rhs, st);
    if (e != cudaSuccess) return set_err(err, err_len, NK_ECUDA, cudaGetErrorString(e));
    nk::launch_inner_lanczos(in, st);
    e = (cudaError_t)nk::launch_rhi(in, st);
    if (e != cudaSuccess) return set_err(err, err_len, NK_ECUDA, cudaGetErrorString(e));
    nk::launch_inner_combine(in, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(err, err_len, NK_ECUDA, cudaGetErrorString(e));
    int status[kMaxRhs];
    e = cudaMemcpyAsync(status, in.status, sizeof(int) * n_rhs, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_err(err, err_len, NK_ECUDA, cudaGetErrorString(e));
    for (int r = 0; r < n_rhs; ++r) {
        switch (status[r]) {
            case nk::kStatusOK:
            case nk::kStatusZeroSource: break;
            case nk::kStatusBreakdown:
            case nk::kStatusInnerBreakdown:
                return set_err(err, err_len, NK_EBREAKDOWN, "inner two-sided Lanczos: serious breakdown");
            case nk::kStatusRhi:
            case nk::kStatusLU:
                return set_err(err, err_len, NK_ERHI, "Roberts-Higham did not converge or p H_k is singular");
            default:
                return set_err(err, err_len, NK_ECUDA, "unexpected per-RHS status code");
        }
    }
    return set_err(err, err_len, NK_OK, "no error");
}
