// Host engine and C ABI (include/nksign.h): context, device workspace,
// the host code that sequences the kernels of one nested Krylov-Ritz
// evaluation, and CUDA-graph capture of whole solves.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <cstdint>
#include <map>
#include <string>
#include <tuple>
#include <vector>
#include <numeric>

#include "tridiag_eig.h"

#include "../../include/nksign.h"
#include "nk_kernels.h"

using nk::Geom;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Multi-level nesting (Sec. 4.5): sizes of the inner levels below the first.
struct Nesting {
    int n = 0;
    int ell[NK_MAX_LEVELS - 1] = {0};
    long code() const {
        long h = n;
        for (int i = 0; i < n; ++i) h = h * 1031 + ell[i];
        return h;
    }
};

struct GraphKey {
    const void* b;
    void* y;
    int n_rhs, k, ell, j0, j1;
    unsigned flags;
    double p, mu, mw;
    int overlap;
    long nest;
    bool operator<(const GraphKey& o) const {
        return std::tie(b, y, n_rhs, k, ell, j0, j1, flags, p, mu, mw, overlap, nest) <
               std::tie(o.b, o.y, o.n_rhs, o.k, o.ell, o.j0, o.j1, o.flags, o.p, o.mu, o.mw, o.overlap, o.nest);
    }
};

struct nk_ctx {
    int dims[4];
    int V;
    long N;
    int antiperiodic;
    int device;
    double mu = 0.0, m_w = 0.0;
    bool mu_set = false;
    int j0 = -1;
    int j1 = -1;   // first outer step whose recurrence runs in two-float arithmetic (< 0: none)
    Nesting nest;  // levels below the first (nk_set_nesting)
    int adapt_start = 0;   // adaptive k: first check (0: NK_ADAPT_FIRST(l))
    bool links = false;
    double2* U64 = nullptr;
    float2* U32 = nullptr;
    nk::dfc* Udf = nullptr;   // two-float links for the early stencil steps of NK_MIXED
    DevBuf ws;            // solve workspace (carved per solve shape)
    DevBuf staging;       // host-pointer API: device copies of b and y
    DevBuf links_tmp;
    DevBuf inner_tmp;     // nk_inner_sign / nk_features scratch (never the staged b and y)
    DevBuf eps_buf;       // NK_EPS_EST: approx(approx(x)) and the per-RHS sums
    // LR deflation (nk_set_deflation): m eigenpairs, right and left vectors
    // [m][12 V] (ABI layout), -1 and sgn(Re lambda_i) per pair, the gap
    int defl_m = 0;
    double2* defl_R = nullptr;
    double2* defl_L = nullptr;   // == defl_R when no left vectors were given
    double* defl_neg = nullptr;
    double* defl_sgn = nullptr;
    double defl_gap = 0.0;
    DevBuf defl_buf;      // x_minus and the coefficients <l_i, b_r>
    DevBuf cg_buf;        // nk_overlap_solve: the CG vectors
    // phase events recorded inside every solve (captured into its graph):
    // end of the outer basis, end of the inner part, start of an adaptive chunk
    cudaEvent_t ph[3] = {nullptr, nullptr, nullptr};
    nk_mlp* predictor = nullptr;   // NK_PREDICT (not owned)
    // exec, kernels per replay; at most kMaxGraphs (a caller cycling through
    // buffers would otherwise instantiate one graph per pair)
    std::map<GraphKey, std::pair<cudaGraphExec_t, int>> graphs;
    std::map<std::tuple<int, int, int>, nk_launch> tune;  // (n_rhs, two_sided, mixed) -> launch shape
    struct Pending {                 // an NK_ASYNC solve not yet collected
        bool on = false;
        cudaStream_t st = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        int n_rhs = 0, k = 0, ell = 0, launches = 0;
        const int *status = nullptr, *iters = nullptr;
        const double *p = nullptr, *zmin = nullptr, *zmax = nullptr, *xnorm = nullptr;
    } pending;
    std::string err = "no error";
};

namespace {

int fail(nk_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(nk_ctx* c, cudaError_t e, const char* what) {
    return fail(c, NK_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define NK_CUDA(ctx, call)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

int ensure(nk_ctx* c, DevBuf& b, size_t bytes) {
    if (b.bytes >= bytes) return NK_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    // graphs hold pointers into the old workspace
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.second.first);
    c->graphs.clear();
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, NK_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                      cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return NK_OK;
}

// Records a phase event on st.  Under stream capture a plain record only
// orders the captured work; cudaEventRecordExternal makes the graph record the
// event when it runs, so that the phase times can be read afterwards.
void record_phase(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    cudaEventRecordWithFlags(e, st, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                       : cudaEventRecordDefault);
}

// Elapsed milliseconds between two recorded events; a failed query (an event
// not recorded) gives 0 and leaves no pending error behind.
double elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return ms;
}

void clear_graph_cache(nk_ctx* c) {
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.second.first);
    c->graphs.clear();
}

Geom geom_of(const nk_ctx* c) {
    Geom g;
    g.Lx = c->dims[0]; g.Ly = c->dims[1]; g.Lz = c->dims[2]; g.Lt = c->dims[3];
    g.V = c->V;
    g.antiperiodic = c->antiperiodic;
    return g;
}

double kappa_of(const nk_ctx* c) { return 1.0 / (8.0 + 2.0 * c->m_w); }

// Carves the solve workspace; returns total bytes (dry run when base == nullptr).
struct Layout {
    nk::Outer o;
    nk::Inner in;
    nk::Inner deeper[NK_MAX_LEVELS - 1];   // multi-level nesting: buffers of the levels below the first
    int n_deeper;
    double2* y_soa;
    double2* cp;      // lift coefficients c'_j, [rhs][k]
    double2* c_prev;  // adaptive k: c of the previous check (finally the accepted c), [rhs][k]
    double2* dn;      // adaptive k: (|c - c_prev|, |c|) per RHS
    int* kused;       // basis vectors that enter the lift, per RHS
    size_t total;
};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

Layout carve(char* base, const Geom& g, int n_rhs, int k, int ell, bool two_sided, bool double_pass,
             const nk_launch& lc, bool mixed, const Nesting& nest = Nesting(), bool full_left = false) {
    const int nblk = lc.step2_blocks;
    Layout L;
    std::memset(&L, 0, sizeof(L));
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += align_up(bytes);
        return p;
    };
    const long N = 12L * g.V;
    const size_t vec = (size_t)N * sizeof(double2);
    L.y_soa = (double2*)take(vec * n_rhs);
    nk::Outer& o = L.o;
    o.N = N; o.n_rhs = n_rhs; o.k = k; o.nblk = nblk; o.two_sided = two_sided;
    o.st_threads = lc.stencil_threads;
    o.st_order = lc.stencil_order;
    o.st_threads_df = lc.early_threads;
    o.st_order_df = lc.early_order;
    o.st_split = lc.stencil_split;
    o.st_split_df = lc.early_split;
    o.npart = std::max(nblk, nk::dslash_step1_blocks(g, std::min(lc.stencil_threads, lc.early_threads)));
    o.npart = std::max(o.npart, nk::stencil32_blocks(g, two_sided ? 2 * n_rhs : n_rhs));
    o.q_ring = double_pass ? 1 : 0;
    o.qcols = double_pass ? 3 : k + 1;   // single pass: k basis vectors + one scratch column
    o.Q = (double2*)take(vec * (size_t)o.qcols * n_rhs);
    o.pcols = full_left ? k + 1 : 3;
    if (two_sided) o.P = (double2*)take(vec * (size_t)o.pcols * n_rhs);
    o.q32 = (float4*)take((size_t)N * sizeof(float2) * n_rhs);    // pair layout: N / 2 float4 per RHS
    if (two_sided) o.p32 = (float4*)take((size_t)N * sizeof(float2) * n_rhs);
    if (mixed) o.s32 = (float4*)take((size_t)N * sizeof(float2) * n_rhs * (two_sided ? 2 : 1));
    if (mixed) o.s64 = (double2*)take(vec * n_rhs * (two_sided ? 2 : 1));
    o.qdf = (nk::dfc*)take((size_t)N * 16 * n_rhs);
    if (two_sided) o.pdf = (nk::dfc*)take((size_t)N * 16 * n_rhs);
    o.q_df_from = 1 << 30;
    o.ring_from = 1 << 30;
    if (mixed) {
        o.qr = (nk::dfc*)take((size_t)N * 16 * 3 * n_rhs);
        if (two_sided) o.pr = (nk::dfc*)take((size_t)N * 16 * 3 * n_rhs);
    }
    o.alpha = (double2*)take(sizeof(double2) * (size_t)k * n_rhs);
    o.beta = (double2*)take(sizeof(double2) * (size_t)k * n_rhs);
    o.gamma = (double2*)take(sizeof(double2) * (size_t)k * n_rhs);
    o.partials = (double2*)take(sizeof(double2) * (size_t)o.npart * n_rhs);
    o.counters = (unsigned*)take(sizeof(unsigned) * n_rhs);
    o.sc = (double2*)take(sizeof(double2) * nk::kScalars * n_rhs);
    o.status = (int*)take(sizeof(int) * n_rhs);
    o.xnorm = (double*)take(sizeof(double) * n_rhs);
    L.cp = (double2*)take(sizeof(double2) * (size_t)k * n_rhs);
    nk::Inner& in = L.in;
    in.n_rhs = n_rhs; in.k = k; in.ell = ell; in.two_sided = two_sided;
    in.alpha = o.alpha; in.beta = o.beta; in.gamma = o.gamma;
    in.p = (double*)take(sizeof(double) * n_rhs);
    in.zmin = (double*)take(sizeof(double) * n_rhs);
    in.zmax = (double*)take(sizeof(double) * n_rhs);
    in.work = (double2*)take(sizeof(double2) * nk::inner_work_elems(k) * n_rhs);
    in.ipiv = (int*)take(sizeof(int) * (size_t)k * n_rhs);
    in.Vl = (double2*)take(sizeof(double2) * (size_t)ell * k * n_rhs);
    in.al = (double2*)take(sizeof(double2) * (size_t)ell * n_rhs);
    in.bl = (double2*)take(sizeof(double2) * (size_t)ell * n_rhs);
    in.gl = (double2*)take(sizeof(double2) * (size_t)ell * n_rhs);
    in.S = (double2*)take(sizeof(double2) * (size_t)ell * ell * n_rhs);
    in.s = (double2*)take(sizeof(double2) * (size_t)ell * n_rhs);
    in.rhi_iters = (int*)take(sizeof(int) * n_rhs);
    in.c = (double2*)take(sizeof(double2) * (size_t)k * n_rhs);
    L.c_prev = (double2*)take(sizeof(double2) * (size_t)k * n_rhs);
    L.dn = (double2*)take(sizeof(double2) * n_rhs);
    L.kused = (int*)take(sizeof(int) * n_rhs);
    in.status = o.status;
    // levels below the first (sizes clipped to the level above); RHi runs on
    // the deepest, whose S buffer is the only one used
    int kl = ell;
    L.n_deeper = nest.n;
    for (int d = 0; d < nest.n; ++d) {
        nk::Inner& q = L.deeper[d];
        q = in;
        q.k = kl;
        q.kstride = 0;
        q.ell = std::min(nest.ell[d], kl);
        q.p = (double*)take(sizeof(double) * n_rhs);
        q.zmin = (double*)take(sizeof(double) * n_rhs);
        q.zmax = (double*)take(sizeof(double) * n_rhs);
        q.work = (double2*)take(sizeof(double2) * nk::inner_work_elems(q.k) * n_rhs);
        q.ipiv = (int*)take(sizeof(int) * (size_t)q.k * n_rhs);
        q.Vl = (double2*)take(sizeof(double2) * (size_t)q.ell * q.k * n_rhs);
        q.al = (double2*)take(sizeof(double2) * (size_t)q.ell * n_rhs);
        q.bl = (double2*)take(sizeof(double2) * (size_t)q.ell * n_rhs);
        q.gl = (double2*)take(sizeof(double2) * (size_t)q.ell * n_rhs);
        q.S = (double2*)take(sizeof(double2) * (size_t)q.ell * q.ell * n_rhs);
        q.s = (double2*)take(sizeof(double2) * (size_t)q.ell * n_rhs);
        q.rhi_iters = (int*)take(sizeof(int) * n_rhs);
        kl = q.ell;
    }
    // the inner part stays FP64 in every schedule: with a Ritz value of H_k'
    // near the imaginary axis its sign is ill conditioned, and two-float
    // arithmetic there left single sources of the 16^3 x 32 test at 2.5e-8
    in.df_inner = 0;
    in.p_shared = 0;
    L.total = off;
    return L;
}

int blocks_per_rhs(long N, int n_rhs) {
    // fixed per shape and device (deterministic reductions): at least two
    // tiles of sites per CTA of the streaming step kernels, and at most one
    // wave of them over all RHS
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    const long V = N / 12;
    const long need = std::max(1L, V / (2L * nk::stream_tile_sites()));
    const long cap = std::max(1L, (long)sms * nk::stream_ctas_per_sm() / n_rhs);
    return (int)std::min(need, cap);
}

// The launch shape of a solve: the tuned one for (n_rhs, two-sided, mixed),
// else the default (128 sites per CTA, vector-fastest grid, blocks_per_rhs).
nk_launch launch_cfg(const nk_ctx* c, int n_rhs, bool ts, bool mixed) {
    auto it = c->tune.find(std::make_tuple(n_rhs, ts ? 1 : 0, mixed ? 1 : 0));
    if (it != c->tune.end()) return it->second;
    nk_launch d;
    d.stencil_threads = 128;
    d.stencil_order = 0;
    d.step2_blocks = blocks_per_rhs(c->N, n_rhs);
    d.early_threads = 128;
    d.early_order = 0;
    d.stencil_split = 1;
    d.early_split = 1;
    return d;
}

bool valid_launch(const nk_launch& l) {
    auto threads_ok = [](int t) { return t == 64 || t == 128 || t == 256; };
    auto order_ok = [](int o) { return o == 0 || o == 1; };
    auto split_ok = [](int s) { return s == 1 || s == 3; };
    return threads_ok(l.stencil_threads) && order_ok(l.stencil_order) && threads_ok(l.early_threads) &&
           order_ok(l.early_order) && split_ok(l.stencil_split) && split_ok(l.early_split) &&
           l.step2_blocks >= 1 && l.step2_blocks <= 4096;
}

// Entry points that write the context's workspace, links or deflation
// vectors refuse while an NK_ASYNC solve still uses them.
static int busy(nk_ctx* c) {
    return c->pending.on ? fail(c, NK_ESTATE, "an NK_ASYNC solve is pending on this context: nk_wait first")
                         : NK_OK;
}

int check_solve_args(nk_ctx* c, int n_rhs, int k, int ell, double tol) {
    if (!c) return NK_EINVAL;
    if (int rb = busy(c)) return rb;
    if (!c->links) return fail(c, NK_ESTATE, "no links loaded (nk_load_links)");
    if (!c->mu_set) return fail(c, NK_ESTATE, "mu and m_w not set (nk_set_mu_mw)");
    if (n_rhs < 1 || n_rhs > NK_MAX_RHS) return fail(c, NK_EINVAL, "n_rhs must be in [1, 12]");
    if (k < 2 || (k & 1)) return fail(c, NK_EINVAL, "k must be even and >= 2");
    if (ell < 2 || (ell & 1)) return fail(c, NK_EINVAL, "l must be even and >= 2");
    if (ell > k) return fail(c, NK_EINVAL, "l must not exceed k");
    if (ell > 256) return fail(c, NK_EINVAL, "l must not exceed 256");
    if (k > nk::kMaxInnerK) return fail(c, NK_EINVAL, "k must not exceed 1536");
    if (!(tol >= 0.0) || !(tol < 1.0)) return fail(c, NK_EINVAL, "tol must be in [0, 1)");
    return NK_OK;
}

// Sequences launches on one stream; counts them and, in NK_PROFILE mode,
// brackets each with CUDA events recorded on that stream.
struct Launcher {
    cudaStream_t st;
    bool profile = false;
    int launches = 0;
    int n_class[NK_NCLASS] = {0};
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
    template <typename F>
    void run(int cls, int nkernels, F&& f) {
        run_counted(cls, [&] {
            f();
            return nkernels;
        });
    }
    // f returns the number of kernels it launched
    template <typename F>
    void run_counted(int cls, F&& f) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (profile) {
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, st);
        }
        const int nkernels = f();
        if (profile) {
            cudaEventRecord(b, st);
            marks.push_back({cls, {a, b}});
        }
        launches += nkernels;
        n_class[cls] += nkernels;
    }
    void collect(double* t_ms) {
        for (auto& m : marks) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, m.second.first, m.second.second);
            t_ms[m.first] += ms;
            cudaEventDestroy(m.second.first);
            cudaEventDestroy(m.second.second);
        }
        marks.clear();
    }
};

// The stencil precision of outer step j: FP64 (NK_FP64); in the mixed
// schedule the two-float stencil (or, with NK_PREFIX_FP64, the FP64 one)
// before step j0 and FP32 from j0 on.
struct Schedule {
    bool mixed = false;
    bool prefix64 = false;
    int j0 = 0;
    int prec(int j) const { return !mixed ? 64 : (j < j0 ? (prefix64 ? 64 : 48) : 32); }
};

// The copy of the new vectors that the stencil of step j reads: none for the
// FP64 stencil, FP32 for the FP32 one; a two-float stencil reads the rings.
int copy_mode_for(const Schedule& s, int j) {
    const int p = s.prec(j);
    return p == 32 ? nk::kCopy32 : (p == 48 ? nk::kCopyDF : nk::kCopyNone);
}

void enqueue_outer_init(const nk::Outer& o, const Schedule& s, Launcher& L, bool keep_status = false) {
    cudaStream_t st = L.st;
    L.run(NK_CLASS_OTHER, 2, [&] { nk::launch_outer_init(o, copy_mode_for(s, 0), st, keep_status); });
}

// steps j in [j_begin, j_end); step 2 runs for every step but the last of the
// whole recurrence (j = o.k - 1).  Mixed schedule: steps j >= o.ring_from run
// the recurrence in two-float arithmetic on the rings (the optional two-float
// recurrence); an FP64 step 2 stores two-float copies of its new vectors only
// when a two-float stencil (the next step) or a ring step (from ring_from - 1
// on, the previous vector of the first ring step) reads them.
void enqueue_outer_steps(nk_ctx* c, const nk::Outer& o, const Schedule& s, int j_begin, int j_end, Launcher& L) {
    const Geom g = geom_of(c);
    const double kap = kappa_of(c);
    cudaStream_t st = L.st;
    for (int j = j_begin; j < j_end; ++j) {
        const int prec = s.prec(j);
        const void* U = prec == 64 ? (const void*)c->U64 : (prec == 48 ? (const void*)c->Udf : (const void*)c->U32);
        const int cls = prec == 64 ? NK_CLASS_DSLASH64 : (prec == 48 ? NK_CLASS_DSLASH_DF : NK_CLASS_DSLASH);
        if (nk::split_step(prec, o, j)) {
            // the stencil, then the FP64 step-1 kernel, timed with the FP64 recurrence
            L.run(cls, 1, [&] { nk::launch_stencil_step(prec, U, g, o, j, kap, c->mu, st); });
            L.run(NK_CLASS_STEP2, 1, [&] { nk::launch_outer_step1(o, j, prec == 48, st); });
        } else {
            L.run_counted(cls, [&] { return nk::launch_dslash_step1(prec, U, g, o, j, kap, c->mu, st); });
        }
        if (j < o.k - 1) {
            const bool ring = s.mixed && j >= o.ring_from;
            const bool write_ring = s.mixed && (s.prec(j + 1) == 48 || j + 1 >= o.ring_from - 1);
            L.run(ring ? NK_CLASS_STEP2_DF : NK_CLASS_STEP2, 1, [&] {
                nk::launch_outer_step2(o, j, copy_mode_for(s, j + 1), ring, write_ring, st);
            });
        }
    }
}

void enqueue_outer(nk_ctx* c, const nk::Outer& o, const Schedule& s, Launcher& L, int steps = -1,
                   bool keep_status = false) {
    enqueue_outer_init(o, s, L, keep_status);
    enqueue_outer_steps(c, o, s, 0, steps < 0 ? o.k : steps, L);
}

// b (ABI layout, device) -> q_0 of every RHS
void enqueue_load_sources(nk_ctx* c, const nk::Outer& o, const double* b_dev, int n_rhs, Launcher& L) {
    const long qs = (long)o.qcols * c->N;
    L.run(NK_CLASS_OTHER, 1, [&] {
        nk::launch_abi_to_soa((const double2*)b_dev, c->N, nk::outer_q(o, 0, 0), qs, c->V, n_rhs, L.st);
    });
}

int effective_j0(const nk_ctx* c, int k) { return c->j0 < 0 ? k / 4 : std::min(c->j0, k); }
// first step of the two-float recurrence; none (FP64 throughout) unless set
int effective_j1(const nk_ctx* c) { return c->j1 < 0 ? (1 << 30) : c->j1; }

Schedule schedule_of(const nk_ctx* c, unsigned flags, int k) {
    Schedule s;
    s.mixed = (flags & NK_MIXED) != 0;
    s.prefix64 = (flags & NK_PREFIX_FP64) != 0;
    s.j0 = effective_j0(c, k);
    return s;
}

// The inner part of App. C steps 3-6 from the first level `in1` (its H is
// the outer H_k): with multi-level nesting (Sec. 4.5) each level below runs
// steps 3-4 on the Ritz matrix of the level above (its own p by Eq. popt),
// RHi runs on the deepest Ritz matrix, and c = V_l1 V_l2 ... s is lifted back
// level by level into in1.c.  *iters: the RHi counts (of the deepest level).
cudaError_t enqueue_inner_chain(const Layout& Lw, const nk::Inner& in1, Launcher& L, const int** iters = nullptr) {
    cudaStream_t st = L.st;
    nk::Inner lv[NK_MAX_LEVELS];
    lv[0] = in1;
    int n = 1;
    for (int d = 0; d < Lw.n_deeper; ++d, ++n) {
        nk::Inner q = Lw.deeper[d];
        const nk::Inner& up = lv[n - 1];
        q.n_rhs = up.n_rhs;
        q.two_sided = up.two_sided;
        q.status = up.status;
        q.alpha = up.al;
        q.beta = up.bl;
        q.gamma = up.gl;
        q.k = up.ell;
        q.kstride = 0;
        q.ell = std::min(Lw.deeper[d].ell, q.k);
        q.p_fixed = 0.0;
        q.p_shared = 0;
        q.c = up.s;   // the lift of this level lands in the s of the level above
        lv[n] = q;
    }
    for (int i = 0; i < n; ++i)
        L.run(NK_CLASS_INNER, nk::inner_launches(lv[i]), [&] { nk::launch_inner_lanczos(lv[i], st); });
    cudaError_t e = cudaSuccess;
    L.run(NK_CLASS_RHI, 1, [&] { e = (cudaError_t)nk::launch_rhi(lv[n - 1], st); });
    if (e != cudaSuccess) return e;
    for (int i = n - 1; i >= 1; --i) L.run(NK_CLASS_INNER, 1, [&] { nk::launch_inner_combine(lv[i], st); });
    if (iters) *iters = lv[n - 1].rhi_iters;
    return cudaSuccess;
}

// Enqueues a whole solve (device pointers in ABI layout). Returns cudaError_t of launches.
cudaError_t enqueue_solve(nk_ctx* c, Layout& Lw, const double* b_dev, double* y_dev, int n_rhs,
                          double p, unsigned flags, bool overlap, Launcher& L) {
    const bool mixed = (flags & NK_MIXED) != 0;
    const bool dp = (flags & NK_DOUBLE_PASS) != 0;
    const Schedule sch = schedule_of(c, flags, Lw.o.k);
    cudaStream_t st = L.st;
    nk::Outer o = Lw.o;
    if (mixed) o.ring_from = effective_j1(c);
    if (mixed && o.qr && !o.q_ring) o.q_df_from = o.ring_from + 1;   // written by the two-float step 2
    nk::Inner in = Lw.in;
    in.p_fixed = p;
    in.p_shared = (flags & NK_SHARED_P) ? 1 : 0;
    enqueue_load_sources(c, o, b_dev, n_rhs, L);
    L.run(NK_CLASS_OTHER, 1, [&] { nk::launch_fill_int(Lw.kused, n_rhs, o.k, st); });
    enqueue_outer(c, o, sch, L);
    record_phase(c->ph[0], st);   // the outer basis is complete
    cudaError_t e = enqueue_inner_chain(Lw, in, L);
    if (e != cudaSuccess) return e;
    record_phase(c->ph[1], st);   // the inner part is complete
    L.run(NK_CLASS_LIFT, 2, [&] {
        nk::launch_inner_combine(in, st);
        nk::launch_lift_coef(o, in.c, Lw.kused, Lw.cp, st);
    });
    if (dp) {
        // second pass: regenerate the identical basis and accumulate y = sum_j c'_j q_j
        o.y = Lw.y_soa;
        o.cp = Lw.cp;
        cudaMemsetAsync(Lw.y_soa, 0, sizeof(double2) * (size_t)c->N * n_rhs, st);
        enqueue_load_sources(c, o, b_dev, n_rhs, L);
        enqueue_outer(c, o, sch, L, -1, true);
    }
    L.run(NK_CLASS_LIFT, 1, [&] { nk::launch_lift(o, Lw.cp, Lw.kused, Lw.y_soa, st); });
    L.run(NK_CLASS_OTHER, 1, [&] {
        nk::launch_soa_to_abi(Lw.y_soa, c->N, (double2*)y_dev, c->N, overlap ? (const double2*)b_dev : nullptr,
                              c->N, c->V, n_rhs, st);
    });
    return cudaGetLastError();
}

// Adaptive k (tol > 0): the outer recurrence runs in chunks; at each check the
// inner part gives c = V_l sgn(H_l) e_1 from the current H_k (the leading k x k
// block), and a RHS is frozen at that k once |c - c_prev| <= tol |c| at two
// consecutive checks.  Launched kernel by kernel (host decisions between chunks).
cudaError_t solve_adaptive(nk_ctx* c, Layout& Lw, const double* b_dev, double* y_dev, int n_rhs, int kmax, int ell,
                           double tol, double p, unsigned flags, bool overlap, Launcher& L,
                           std::vector<int>& kused_h, std::vector<int>& notconv, int& checks, double tph[2]) {
    cudaStream_t st = L.st;
    const bool mixed = (flags & NK_MIXED) != 0;
    const Schedule sch = schedule_of(c, flags, kmax);
    nk::Outer o = Lw.o;
    if (mixed) o.ring_from = effective_j1(c);
    if (mixed && o.qr && !o.q_ring) o.q_df_from = o.ring_from + 1;
    nk::Inner in = Lw.in;
    in.p_fixed = p;
    in.p_shared = (flags & NK_SHARED_P) ? 1 : 0;
    in.kstride = kmax;
    enqueue_load_sources(c, o, b_dev, n_rhs, L);
    enqueue_outer_init(o, sch, L);
    cudaMemsetAsync(Lw.c_prev, 0, sizeof(double2) * (size_t)kmax * n_rhs, st);
    int first = c->adapt_start > 0 ? c->adapt_start : NK_ADAPT_FIRST(ell);
    first = std::max(2, std::min(kmax, first + (first & 1)));
    std::vector<int> hits(n_rhs, 0), frozen(n_rhs, 0), status(n_rhs, 0);
    std::vector<double2> dn(n_rhs);
    kused_h.assign(n_rhs, kmax);
    notconv.assign(n_rhs, 1);
    checks = 0;
    int j = 0, kc = first;
    while (true) {
        record_phase(c->ph[2], st);
        enqueue_outer_steps(c, o, sch, j, kc, L);
        record_phase(c->ph[0], st);
        nk::Inner ic = in;
        ic.k = kc;
        ic.ell = std::min(ell, kc);
        cudaError_t e = enqueue_inner_chain(Lw, ic, L);
        if (e != cudaSuccess) return e;
        L.run(NK_CLASS_LIFT, 1, [&] { nk::launch_inner_combine(ic, st); });
        L.run(NK_CLASS_OTHER, 1, [&] { nk::launch_adapt_delta(o, in.c, Lw.c_prev, kc, Lw.dn, st); });
        record_phase(c->ph[1], st);
        e = cudaMemcpyAsync(dn.data(), Lw.dn, sizeof(double2) * n_rhs, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(status.data(), o.status, sizeof(int) * n_rhs, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        tph[0] += elapsed_ms(c->ph[2], c->ph[0]);
        tph[1] += elapsed_ms(c->ph[0], c->ph[1]);
        ++checks;
        bool all = true, changed = false;
        for (int r = 0; r < n_rhs; ++r) {
            if (frozen[r]) continue;
            const bool inner_failed = status[r] == nk::kStatusRhi || status[r] == nk::kStatusLU ||
                                      status[r] == nk::kStatusInnerBreakdown;
            if (inner_failed && kc < kmax) {
                // the inner part failed on this H_k (e.g. a Ritz value near the
                // imaginary axis): a failed check; the outer recurrence goes on
                status[r] = nk::kStatusOK;
                hits[r] = 0;
                changed = true;
                all = false;
                continue;
            }
            if (status[r] != nk::kStatusOK) {   // zero source or failure: nothing more to do
                frozen[r] = 1;
                kused_h[r] = kc;
                notconv[r] = 0;
                continue;
            }
            const double rel = dn[r].y > 0.0 ? dn[r].x / dn[r].y : 0.0;
            hits[r] = rel <= tol ? hits[r] + 1 : 0;
            if (hits[r] >= 2) {
                frozen[r] = 1;
                kused_h[r] = kc;
                notconv[r] = 0;
                status[r] = nk::kStatusConverged;
                changed = true;
            } else {
                all = false;
            }
        }
        if (all || kc >= kmax) break;
        if (changed) {
            e = cudaMemcpyAsync(o.status, status.data(), sizeof(int) * n_rhs, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return e;
        }
        j = kc;
        kc = std::min(kmax, kc + NK_ADAPT_STEP);
    }
    // frozen RHS rejoin the lift; the accepted c of every RHS is in c_prev
    for (int r = 0; r < n_rhs; ++r)
        if (status[r] == nk::kStatusConverged) status[r] = nk::kStatusOK;
    cudaError_t e = cudaMemcpyAsync(o.status, status.data(), sizeof(int) * n_rhs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Lw.kused, kused_h.data(), sizeof(int) * n_rhs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    record_phase(c->ph[1], st);   // the lift starts here (t_lift: from ph[1] to the end)
    L.run(NK_CLASS_LIFT, 2, [&] {
        nk::launch_lift_coef(o, Lw.c_prev, Lw.kused, Lw.cp, st);
        nk::launch_lift(o, Lw.cp, Lw.kused, Lw.y_soa, st);
    });
    L.run(NK_CLASS_OTHER, 1, [&] {
        nk::launch_soa_to_abi(Lw.y_soa, c->N, (double2*)y_dev, c->N, overlap ? (const double2*)b_dev : nullptr,
                              c->N, c->V, n_rhs, st);
    });
    return cudaGetLastError();
}

int status_to_code(int s) {
    switch (s) {
        case nk::kStatusOK:
        case nk::kStatusZeroSource: return NK_OK;
        case nk::kStatusBreakdown:
        case nk::kStatusInnerBreakdown: return NK_EBREAKDOWN;
        case nk::kStatusRhi: return NK_ERHI;
        case nk::kStatusLU: return NK_ERHI;
        case nk::kStatusTimeout: return NK_ETIMEOUT;
        default: return NK_ECUDA;
    }
}

// Per-RHS outcome of a finished solve (device arrays read after the stream
// has been synchronised) into codes and stats.
int collect_outcome(nk_ctx* c, int n_rhs, int k_used_max, const std::vector<int>& kused_h,
                    const std::vector<int>& notconv, int checks, int ell, int launches, float ms,
                    const std::vector<int>& status, const std::vector<int>& iters, const std::vector<double>& pv,
                    const std::vector<double>& zmin, const std::vector<double>& zmax, const std::vector<double>& xn,
                    nk_stats* stats) {
    int worst = NK_OK;
    std::vector<int> codes(n_rhs);
    for (int r = 0; r < n_rhs; ++r) {
        codes[r] = status_to_code(status[r]);
        if (codes[r] == NK_OK && notconv[r]) codes[r] = NK_ENOTCONV;
        if (codes[r] != NK_OK && worst == NK_OK) worst = codes[r];
    }
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->n_rhs = n_rhs;
        stats->k_used = k_used_max;
        stats->ell_used = ell;
        stats->checks = checks;
        for (int r = 0; r < n_rhs; ++r) {
            stats->k_rhs[r] = kused_h[r];
            stats->rhi_iters[r] = iters[r];
            stats->status[r] = codes[r];
            stats->p[r] = pv[r];
            stats->z_min[r] = zmin[r];
            stats->z_max[r] = zmax[r];
            stats->xnorm[r] = xn[r];
        }
        stats->t_total_ms = ms;
        stats->launches = launches;
    }
    if (worst == NK_EBREAKDOWN) return fail(c, worst, "two-sided Lanczos: serious breakdown (delta = 0)");
    if (worst == NK_ERHI) return fail(c, worst, "Roberts-Higham iteration did not converge (or p H_k singular)");
    if (worst == NK_ENOTCONV) return fail(c, worst, "adaptive k: tolerance not met at k_max for some RHS");
    return worst;
}

constexpr size_t kMaxGraphs = 16;

// Two CUDA events owned by one solve; destroyed unless handed to a pending
// NK_ASYNC solve (release()).
struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~EventPair() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
    void release() { e0 = e1 = nullptr; }
};

// Device-time split of a finished fixed-k solve from the phase events (graph
// or kernel by kernel): basis, inner part, lift.
void phase_times(const nk_ctx* c, cudaEvent_t e0, cudaEvent_t e1, double out[3]) {
    out[0] = elapsed_ms(e0, c->ph[0]);
    out[1] = elapsed_ms(c->ph[0], c->ph[1]);
    out[2] = elapsed_ms(c->ph[1], e1);
}

// One solve (fixed or adaptive k), sequenced on stream st.
int solve_core(nk_ctx* c, const double* b_dev, int n_rhs, int k, int ell, double tol, double p,
               unsigned flags, double* y_dev, nk_stats* stats, cudaStream_t st, bool overlap) {
    int rc = check_solve_args(c, n_rhs, k, ell, tol);
    if (rc) return rc;
    if (c->pending.on) return fail(c, NK_ESTATE, "an NK_ASYNC solve is pending on this context: nk_wait first");
    const bool async = (flags & NK_ASYNC) != 0;
    if (async && (tol > 0.0 || (flags & NK_PROFILE)))
        return fail(c, NK_EINVAL, "NK_ASYNC needs a fixed k (tol = 0) and no NK_PROFILE");
    const bool adaptive = tol > 0.0;
    const bool dp = (flags & NK_DOUBLE_PASS) != 0;
    if (adaptive && dp) return fail(c, NK_EINVAL, "adaptive k (tol > 0) needs single-pass storage");
    NK_CUDA(c, cudaSetDevice(c->device));
    const bool ts = c->mu != 0.0;
    const nk_launch lc = launch_cfg(c, n_rhs, ts, (flags & NK_MIXED) != 0);
    const bool mixed = (flags & NK_MIXED) != 0;
    Layout dry = carve(nullptr, geom_of(c), n_rhs, k, ell, ts, dp, lc, mixed, c->nest);
    rc = ensure(c, c->ws, dry.total);
    if (rc) return rc;
    Layout Lw = carve((char*)c->ws.p, geom_of(c), n_rhs, k, ell, ts, dp, lc, mixed, c->nest);
    // counters must start at zero; status is (re)set by the norm kernel
    NK_CUDA(c, cudaMemsetAsync(Lw.o.counters, 0, sizeof(unsigned) * n_rhs, st));

    EventPair ev;
    NK_CUDA(c, cudaEventCreate(&ev.e0));
    NK_CUDA(c, cudaEventCreate(&ev.e1));
    NK_CUDA(c, cudaEventRecord(ev.e0, st));
    const bool profile = (flags & NK_PROFILE) != 0;
    const bool use_graph = !adaptive && (flags & (NK_NO_GRAPH | NK_PROFILE)) == 0;
    Launcher L;
    L.st = st;
    L.profile = profile;
    std::vector<int> kused_h(n_rhs, k), notconv(n_rhs, 0);
    int checks = 0;
    double tph[3] = {0.0, 0.0, 0.0};
    if (adaptive) {
        cudaError_t e = solve_adaptive(c, Lw, b_dev, y_dev, n_rhs, k, ell, tol, p, flags, overlap, L, kused_h,
                                       notconv, checks, tph);
        if (e != cudaSuccess) return cuda_fail(c, e, "adaptive solve");
    } else if (use_graph) {
        GraphKey key{b_dev, y_dev, n_rhs, k, ell, c->j0, c->j1, flags, p, c->mu, c->m_w, overlap ? 1 : 0,
                     c->nest.code()};
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            if (c->graphs.size() >= kMaxGraphs) clear_graph_cache(c);
            cudaStream_t cs;
            NK_CUDA(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            NK_CUDA(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            Launcher Lc;
            Lc.st = cs;
            cudaError_t e = enqueue_solve(c, Lw, b_dev, y_dev, n_rhs, p, flags, overlap, Lc);
            cudaGraph_t graph;
            cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            cudaStreamDestroy(cs);
            if (e != cudaSuccess) return cuda_fail(c, e, "enqueue_solve (capture)");
            if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
            cudaGraphExec_t exec;
            cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e3 != cudaSuccess) return cuda_fail(c, e3, "cudaGraphInstantiate");
            it = c->graphs.emplace(key, std::make_pair(exec, Lc.launches)).first;
        }
        NK_CUDA(c, cudaGraphLaunch(it->second.first, st));
        L.launches = it->second.second;
    } else {
        cudaError_t e = enqueue_solve(c, Lw, b_dev, y_dev, n_rhs, p, flags, overlap, L);
        if (e != cudaSuccess) return cuda_fail(c, e, "enqueue_solve");
    }
    NK_CUDA(c, cudaEventRecord(ev.e1, st));
    if (async) {   // collected by nk_wait
        nk_ctx::Pending& P = c->pending;
        P.on = true;
        P.st = st;
        P.e0 = ev.e0;
        P.e1 = ev.e1;
        ev.release();
        P.n_rhs = n_rhs;
        P.k = k;
        P.ell = ell;
        P.launches = L.launches;
        P.status = Lw.o.status;
        P.iters = Lw.n_deeper ? Lw.deeper[Lw.n_deeper - 1].rhi_iters : Lw.in.rhi_iters;
        P.p = Lw.in.p;
        P.zmin = Lw.in.zmin;
        P.zmax = Lw.in.zmax;
        P.xnorm = Lw.o.xnorm;
        return NK_OK;
    }
    // read back per-RHS outcome
    std::vector<int> status(n_rhs), iters(n_rhs);
    std::vector<double> pv(n_rhs), zmin(n_rhs), zmax(n_rhs), xn(n_rhs);
    NK_CUDA(c, cudaMemcpyAsync(status.data(), Lw.o.status, sizeof(int) * n_rhs, cudaMemcpyDeviceToHost, st));
    const int* iters_dev = Lw.n_deeper ? Lw.deeper[Lw.n_deeper - 1].rhi_iters : Lw.in.rhi_iters;
    NK_CUDA(c, cudaMemcpyAsync(iters.data(), iters_dev, sizeof(int) * n_rhs, cudaMemcpyDeviceToHost, st));
    NK_CUDA(c, cudaMemcpyAsync(pv.data(), Lw.in.p, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost, st));
    NK_CUDA(c, cudaMemcpyAsync(zmin.data(), Lw.in.zmin, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost, st));
    NK_CUDA(c, cudaMemcpyAsync(zmax.data(), Lw.in.zmax, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost, st));
    NK_CUDA(c, cudaMemcpyAsync(xn.data(), Lw.o.xnorm, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost, st));
    NK_CUDA(c, cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.e0, ev.e1);
    if (adaptive) {
        tph[2] = elapsed_ms(c->ph[1], ev.e1);
    } else {
        phase_times(c, ev.e0, ev.e1, tph);
    }
    double tcm[NK_NCLASS] = {0};   // NK_PROFILE: summed device time per class
    int ncl[NK_NCLASS] = {0};
    if (profile) {
        L.collect(tcm);
        for (int q = 0; q < NK_NCLASS; ++q) ncl[q] = L.n_class[q];
    }
    rc = collect_outcome(c, n_rhs, *std::max_element(kused_h.begin(), kused_h.end()), kused_h, notconv, checks, ell,
                         L.launches, ms, status, iters, pv, zmin, zmax, xn, stats);
    if (stats) {
        stats->t_basis_ms = tph[0];
        stats->t_inner_ms = tph[1];
        stats->t_lift_ms = tph[2];
        if (profile) {
            std::memcpy(stats->t_class_ms, tcm, sizeof(tcm));
            for (int q = 0; q < NK_NCLASS; ++q) stats->n_class[q] = ncl[q];
        }
    }
    return rc;
}

// NK_PREDICT: predict (k, l) from source 0 (nk_predict_sizes), then the
// adaptive solve from the predicted start, repeated once with the caller's l
// if the tolerance is not met with the predicted one.
int predicted_solve(nk_ctx* c, const double* b_dev, int n_rhs, int k, int ell, double tol, double p, unsigned flags,
                    double* y_dev, nk_stats* S, cudaStream_t st, bool overlap) {
    if (!(flags & NK_PREDICT)) return solve_core(c, b_dev, n_rhs, k, ell, tol, p, flags, y_dev, S, st, overlap);
    if (!(tol > 0.0)) return fail(c, NK_EINVAL, "NK_PREDICT needs adaptive k (tol > 0)");
    if (!c->predictor) return fail(c, NK_ESTATE, "NK_PREDICT: no predictor (nk_set_predictor)");
    int rc = check_solve_args(c, n_rhs, k, ell, tol);
    if (rc) return rc;
    int kp = 0, lp = 0;
    rc = nk_predict_sizes(c, c->predictor, b_dev, k, &kp, &lp, (void*)st);
    if (rc) return rc;
    // l too small never passes the test: a margin of 1.5 (the inner part
    // costs O(k l), little against a repeated solve)
    int l_use = 2 * (int)std::ceil(0.75 * lp);
    l_use = std::max(2, std::min(std::min(l_use, kp), std::min(256, k)));
    l_use -= l_use & 1;
    const unsigned f = flags & ~NK_PREDICT;
    const int saved = c->adapt_start;
    c->adapt_start = std::max(64, kp - 2 * NK_ADAPT_STEP);
    rc = solve_core(c, b_dev, n_rhs, k, l_use, tol, p, f, y_dev, S, st, overlap);
    c->adapt_start = saved;
    int fallback = 0;
    if (rc == NK_ENOTCONV && l_use < ell) {
        const double t_first = S->t_total_ms;
        rc = solve_core(c, b_dev, n_rhs, k, ell, tol, p, f, y_dev, S, st, overlap);
        S->t_total_ms += t_first;
        fallback = 1;
    }
    S->k_pred = kp;
    S->ell_pred = lp;
    S->predict_fallback = fallback;
    return rc;
}

bool solve_failed_hard(int rc) { return rc != NK_OK && rc != NK_EBREAKDOWN && rc != NK_ERHI && rc != NK_ENOTCONV; }

// LR deflation (App. C steps 1 and 6) around a solve: the Krylov part runs on
// x_minus = b - sum_i <l_i, b> r_i, and sum_i sgn(lambda_i) <l_i, b> r_i is
// added to its result; D_ov then applies b + gamma5 y to the whole of it.
int deflated_solve(nk_ctx* c, const double* b_dev, int n_rhs, int k, int ell, double tol, double p, unsigned flags,
                   double* y_dev, nk_stats* S, cudaStream_t st, bool overlap) {
    const int m = c->defl_m;
    if (m == 0) return predicted_solve(c, b_dev, n_rhs, k, ell, tol, p, flags, y_dev, S, st, overlap);
    int rc = check_solve_args(c, n_rhs, k, ell, tol);
    if (rc) return rc;
    NK_CUDA(c, cudaSetDevice(c->device));
    const size_t vb = align_up(sizeof(double2) * (size_t)c->N * n_rhs);
    rc = ensure(c, c->defl_buf, vb + sizeof(double2) * (size_t)m * NK_MAX_RHS);
    if (rc) return rc;
    double2* xm = (double2*)c->defl_buf.p;
    double2* d = (double2*)((char*)c->defl_buf.p + vb);
    nk::launch_defl_dots(c->defl_L, (const double2*)b_dev, c->N, m, n_rhs, d, st);
    nk::launch_defl_axpy((const double2*)b_dev, xm, c->defl_R, d, c->defl_neg, c->N, m, n_rhs, st);
    NK_CUDA(c, cudaGetLastError());
    rc = predicted_solve(c, (const double*)xm, n_rhs, k, ell, tol, p, flags, y_dev, S, st, false);
    if (solve_failed_hard(rc)) return rc;
    nk::launch_defl_axpy((const double2*)y_dev, (double2*)y_dev, c->defl_R, d, c->defl_sgn, c->N, m, n_rhs, st);
    if (overlap) nk::launch_overlap_finish((const double2*)b_dev, (double2*)y_dev, c->N, n_rhs, st);
    NK_CUDA(c, cudaGetLastError());
    if (!(flags & NK_ASYNC)) NK_CUDA(c, cudaStreamSynchronize(st));
    S->defl_m = m;
    S->defl_gap = c->defl_gap;
    return rc;
}

// NK_EPS_EST: the error estimate of Sec. 3 for every RHS: x~ = approx(y) with
// y = approx(x), eps = |x~ - x| / (2|x|).
int eps_estimate(nk_ctx* c, const double* b_dev, const double* y_dev, int n_rhs, int k, int ell, double tol,
                 double p, unsigned flags, cudaStream_t st, nk_stats* stats) {
    const size_t vb = align_up(sizeof(double2) * (size_t)c->N * n_rhs);
    int rc = ensure(c, c->eps_buf, vb + sizeof(double2) * NK_MAX_RHS);
    if (rc) return rc;
    double2* x2 = (double2*)c->eps_buf.p;
    double2* sums = (double2*)((char*)c->eps_buf.p + vb);
    nk_stats s2;
    std::memset(&s2, 0, sizeof(s2));
    rc = deflated_solve(c, y_dev, n_rhs, k, ell, tol, p, flags & ~(NK_EPS_EST | NK_PREDICT | NK_ASYNC), (double*)x2,
                        &s2, st, false);
    if (solve_failed_hard(rc)) return rc;
    nk::launch_eps_sums((const double2*)b_dev, x2, n_rhs, c->N, sums, st);
    NK_CUDA(c, cudaGetLastError());
    std::vector<double2> h(n_rhs);
    NK_CUDA(c, cudaMemcpyAsync(h.data(), sums, sizeof(double2) * n_rhs, cudaMemcpyDeviceToHost, st));
    NK_CUDA(c, cudaStreamSynchronize(st));
    if (stats)
        for (int r = 0; r < n_rhs; ++r)
            stats->eps_sgn2[r] = h[r].y > 0.0 ? std::sqrt(h[r].x) / (2.0 * std::sqrt(h[r].y)) : 0.0;
    return NK_OK;
}

// A solve: optional prediction of (k, l) (NK_PREDICT), optional LR
// deflation (nk_set_deflation), optional error estimate afterwards (NK_EPS_EST).
int solve_dev(nk_ctx* c, const double* b_dev, int n_rhs, int k, int ell, double tol, double p,
              unsigned flags, double* y_dev, nk_stats* stats, cudaStream_t st, bool overlap) {
    if (!c) return NK_EINVAL;
    const bool predict = (flags & NK_PREDICT) != 0;
    const bool eps = (flags & NK_EPS_EST) != 0;
    if ((predict || eps) && (flags & NK_ASYNC)) return fail(c, NK_EINVAL, "NK_PREDICT / NK_EPS_EST need a blocking solve");
    if (eps && overlap) return fail(c, NK_EINVAL, "NK_EPS_EST applies to the sign function, not to D_ov");
    if (!predict && !eps && c->defl_m == 0)
        return solve_core(c, b_dev, n_rhs, k, ell, tol, p, flags, y_dev, stats, st, overlap);
    nk_stats local;
    nk_stats* S = stats ? stats : &local;
    std::memset(S, 0, sizeof(*S));
    int rc = deflated_solve(c, b_dev, n_rhs, k, ell, tol, p, flags & ~NK_EPS_EST, y_dev, S, st, overlap);
    if (solve_failed_hard(rc)) return rc;
    if (eps) {
        // the second application uses the sizes the first one ended with
        const int l2 = S->ell_used > 0 ? S->ell_used : ell;
        const std::string keep_err = c->err;
        const int rc2 = eps_estimate(c, b_dev, y_dev, n_rhs, k, l2, tol, p, flags, st, S);
        if (rc2 != NK_OK) return rc2;
        c->err = keep_err;
    }
    return rc;
}

}  // namespace

extern "C" {

int nk_create_lattice(const int dims[4], int bc_t_antiperiodic, nk_ctx** out) {
    if (!dims || !out) return NK_EINVAL;
    *out = nullptr;
    long V = 1;
    for (int i = 0; i < 4; ++i) {
        if (dims[i] < 2) return NK_EINVAL;
        V *= dims[i];
    }
    if (V > (1L << 28)) return NK_EINVAL;
    nk_ctx* c = new nk_ctx();
    std::memcpy(c->dims, dims, sizeof(c->dims));
    c->V = (int)V;
    c->N = 12 * V;
    c->antiperiodic = bc_t_antiperiodic ? 1 : 0;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return NK_ECUDA;
    }
    nk::init_kernel_attributes();
    cudaGetLastError();
    for (auto& e : c->ph) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            for (auto& f : c->ph)
                if (f) cudaEventDestroy(f);
            delete c;
            return NK_ECUDA;
        }
    }
    *out = c;
    return NK_OK;
}

static int load_links_impl(nk_ctx* c, const double* U, bool host, cudaStream_t st) {
    if (!c || !U) return NK_EINVAL;
    if (int rb = busy(c)) return rb;
    NK_CUDA(c, cudaSetDevice(c->device));
    const size_t n = (size_t)c->V * 36;
    if (!c->U64) {
        NK_CUDA(c, cudaMalloc(&c->U64, n * sizeof(double2)));
        NK_CUDA(c, cudaMalloc(&c->U32, n * sizeof(float2)));
        NK_CUDA(c, cudaMalloc(&c->Udf, n * 16));
    }
    const double2* src = (const double2*)U;
    if (host) {
        int rc = ensure(c, c->links_tmp, n * sizeof(double2));
        if (rc) return rc;
        NK_CUDA(c, cudaMemcpyAsync(c->links_tmp.p, U, n * sizeof(double2), cudaMemcpyHostToDevice, st));
        src = (const double2*)c->links_tmp.p;
    }
    nk::launch_links_to_device_layout(src, c->U64, c->U32, c->Udf, c->V, st);
    NK_CUDA(c, cudaGetLastError());
    NK_CUDA(c, cudaStreamSynchronize(st));
    c->links = true;
    return NK_OK;
}

int nk_load_links(nk_ctx* c, const double* U) { return load_links_impl(c, U, true, 0); }

int nk_load_links_dev(nk_ctx* c, const double* U_dev, void* stream) {
    return load_links_impl(c, U_dev, false, (cudaStream_t)stream);
}

int nk_set_mu_mw(nk_ctx* c, double mu, double m_w) {
    if (!c) return NK_EINVAL;
    if (!(8.0 + 2.0 * m_w > 0.0) || !std::isfinite(mu) || !std::isfinite(m_w))
        return fail(c, NK_EINVAL, "need finite mu, m_w with 8 + 2 m_w > 0");
    if (c->mu != mu || c->m_w != m_w) {
        for (auto& g : c->graphs) cudaGraphExecDestroy(g.second.first);
        c->graphs.clear();
    }
    c->mu = mu;
    c->m_w = m_w;
    c->mu_set = true;
    return NK_OK;
}

int nk_set_precision(nk_ctx* c, int j0) {
    if (!c) return NK_EINVAL;
    c->j0 = j0;
    return NK_OK;
}

int nk_set_df_recurrence(nk_ctx* c, int j1) {
    if (!c) return NK_EINVAL;
    c->j1 = j1;
    return NK_OK;
}

// M v = D_ov(mu) v + m v (dagger = 0) or M^dagger v = gamma5 D_ov(-mu) gamma5 v + m v
// (dagger = 1; D_ov(mu)^dagger = gamma5 D_ov(-mu) gamma5 because
// A(mu)^dagger = A(-mu)), v and out device ABI vectors; tmp scratch.  For -mu
// the deflated eigenpairs of A(mu) serve A(-mu) = A(mu)^dagger with the roles
// of the right and left eigenvectors exchanged (the signs sgn(Re lambda) are
// those of conj(lambda)).
static int overlap_op(nk_ctx* c, const double2* v, double2* out, double2* tmp, int n_rhs, int k, int ell, double tol,
                      unsigned flags, double mass, bool dagger, cudaStream_t st, int* applications) {
    int rc;
    const unsigned f = flags & ~(NK_ASYNC | NK_EPS_EST);
    if (!dagger) {
        rc = solve_dev(c, (const double*)v, n_rhs, k, ell, tol, 0.0, f, (double*)out, nullptr, st, true);
    } else {
        NK_CUDA(c, cudaMemcpyAsync(tmp, v, sizeof(double2) * (size_t)c->N * n_rhs, cudaMemcpyDeviceToDevice, st));
        nk::launch_gamma5(tmp, c->N, n_rhs, st);
        c->mu = -c->mu;
        std::swap(c->defl_R, c->defl_L);
        rc = solve_dev(c, (const double*)tmp, n_rhs, k, ell, tol, 0.0, f, (double*)out, nullptr, st, true);
        std::swap(c->defl_R, c->defl_L);
        c->mu = -c->mu;
        nk::launch_gamma5(out, c->N, n_rhs, st);
    }
    ++*applications;
    if (rc != NK_OK && rc != NK_ENOTCONV) return rc;
    nk::VecCoefs cm, one;
    for (int r = 0; r < 12; ++r) {
        cm.c[r] = make_double2(mass, 0.0);
        one.c[r] = make_double2(1.0, 0.0);
    }
    nk::launch_vlincomb(out, v, c->N, n_rhs, cm, one, st);   // out += m v
    NK_CUDA(c, cudaGetLastError());
    return NK_OK;
}

static int vdots(nk_ctx* c, const double2* a, const double2* b, int n, double2* dev, std::vector<double2>& h,
                 cudaStream_t st) {
    nk::launch_vdot(a, b, c->N, n, dev, st);
    NK_CUDA(c, cudaMemcpyAsync(h.data(), dev, sizeof(double2) * n, cudaMemcpyDeviceToHost, st));
    NK_CUDA(c, cudaStreamSynchronize(st));
    return NK_OK;
}

int nk_overlap_solve(nk_ctx* c, const double* b, int n_rhs, int k, int ell, double tol_sign, unsigned flags,
                     double mass, double tol_cg, int maxit, double* x, int* iters, double* resid) {
    if (!c || !b || !x) return c ? fail(c, NK_EINVAL, "null pointer") : NK_EINVAL;
    int rc = check_solve_args(c, n_rhs, k, ell, tol_sign);
    if (rc) return rc;
    if (!(mass >= 0.0) || !(tol_cg > 0.0) || maxit < 1) return fail(c, NK_EINVAL, "need mass >= 0, tol_cg > 0, maxit >= 1");
    NK_CUDA(c, cudaSetDevice(c->device));
    const size_t vb = align_up(sizeof(double2) * (size_t)c->N * n_rhs);
    rc = ensure(c, c->cg_buf, 8 * vb);
    if (rc) return rc;
    char* base = (char*)c->cg_buf.p;
    double2 *bd = (double2*)base, *xd = (double2*)(base + vb), *r = (double2*)(base + 2 * vb),
            *p = (double2*)(base + 3 * vb), *q = (double2*)(base + 4 * vb), *s = (double2*)(base + 5 * vb),
            *tmp = (double2*)(base + 6 * vb), *dots = (double2*)(base + 7 * vb);
    cudaStream_t st = 0;
    const size_t bytes = sizeof(double2) * (size_t)c->N * n_rhs;
    NK_CUDA(c, cudaMemcpy(bd, b, bytes, cudaMemcpyHostToDevice));
    NK_CUDA(c, cudaMemsetAsync(xd, 0, bytes, st));
    int apps = 0;
    // r = M^dagger b, p = r
    rc = overlap_op(c, bd, r, tmp, n_rhs, k, ell, tol_sign, flags, mass, true, st, &apps);
    if (rc) return rc;
    NK_CUDA(c, cudaMemcpyAsync(p, r, bytes, cudaMemcpyDeviceToDevice, st));
    std::vector<double2> h(n_rhs);
    if ((rc = vdots(c, r, r, n_rhs, dots, h, st))) return rc;
    std::vector<double> rr(n_rhs), rr0(n_rhs);
    std::vector<int> done(n_rhs, 0), its(n_rhs, 0);
    for (int i = 0; i < n_rhs; ++i) {
        rr[i] = rr0[i] = h[i].x;
        done[i] = !(rr0[i] > 0.0);   // b = 0: x = 0
    }
    int it = 0;
    for (; it < maxit; ++it) {
        bool all = true;
        for (int i = 0; i < n_rhs; ++i) all = all && done[i];
        if (all) break;
        // q = M p, alpha = |r|^2 / |q|^2
        if ((rc = overlap_op(c, p, q, tmp, n_rhs, k, ell, tol_sign, flags, mass, false, st, &apps))) return rc;
        if ((rc = vdots(c, q, q, n_rhs, dots, h, st))) return rc;
        nk::VecCoefs ca, cb, na;
        for (int i = 0; i < 12; ++i) ca.c[i] = cb.c[i] = na.c[i] = make_double2(i < n_rhs ? 0.0 : 0.0, 0.0);
        for (int i = 0; i < n_rhs; ++i) {
            const double al = done[i] || !(h[i].x > 0.0) ? 0.0 : rr[i] / h[i].x;
            ca.c[i] = make_double2(al, 0.0);
            na.c[i] = make_double2(-al, 0.0);
            cb.c[i] = make_double2(1.0, 0.0);
        }
        nk::launch_vlincomb(xd, p, c->N, n_rhs, ca, cb, st);          // x += alpha p
        if ((rc = overlap_op(c, q, s, tmp, n_rhs, k, ell, tol_sign, flags, mass, true, st, &apps))) return rc;
        nk::launch_vlincomb(r, s, c->N, n_rhs, na, cb, st);           // r -= alpha M^dagger q
        if ((rc = vdots(c, r, r, n_rhs, dots, h, st))) return rc;
        nk::VecCoefs one, be;
        for (int i = 0; i < 12; ++i) one.c[i] = be.c[i] = make_double2(i < n_rhs ? 1.0 : 0.0, 0.0);
        for (int i = 0; i < n_rhs; ++i) {
            if (done[i]) { be.c[i] = make_double2(1.0, 0.0); continue; }
            const double rn = h[i].x;
            be.c[i] = make_double2(rr[i] > 0.0 ? rn / rr[i] : 0.0, 0.0);
            rr[i] = rn;
            its[i] = it + 1;
            if (std::sqrt(rn / rr0[i]) <= tol_cg) done[i] = 1;
        }
        nk::launch_vlincomb(p, r, c->N, n_rhs, one, be, st);          // p = r + beta p
        NK_CUDA(c, cudaGetLastError());
    }
    NK_CUDA(c, cudaMemcpy(x, xd, bytes, cudaMemcpyDeviceToHost));
    bool all = true;
    for (int i = 0; i < n_rhs; ++i) {
        if (iters) iters[i] = its[i];
        if (resid) resid[i] = rr0[i] > 0.0 ? std::sqrt(rr[i] / rr0[i]) : 0.0;
        all = all && done[i];
    }
    if (!all) return fail(c, NK_ENOTCONV, "overlap CG: tolerance not met within maxit iterations");
    return NK_OK;
}

int nk_set_deflation(nk_ctx* c, int m, const double* lambda, const double* R, const double* L) {
    if (!c) return NK_EINVAL;
    if (int rb = busy(c)) return rb;
    if (m < 0 || m > NK_MAX_DEFL || (m > 0 && (!lambda || !R)))
        return fail(c, NK_EINVAL, "need 0 <= m <= NK_MAX_DEFL, eigenvalues and right eigenvectors");
    NK_CUDA(c, cudaSetDevice(c->device));
    if (c->defl_L && c->defl_L != c->defl_R) cudaFree(c->defl_L);
    if (c->defl_R) cudaFree(c->defl_R);
    if (c->defl_neg) cudaFree(c->defl_neg);
    if (c->defl_sgn) cudaFree(c->defl_sgn);
    c->defl_R = c->defl_L = nullptr;
    c->defl_neg = c->defl_sgn = nullptr;
    c->defl_m = 0;
    c->defl_gap = 0.0;
    if (m == 0) return NK_OK;
    const size_t bytes = sizeof(double2) * (size_t)m * c->N;
    NK_CUDA(c, cudaMalloc(&c->defl_R, bytes));
    NK_CUDA(c, cudaMemcpy(c->defl_R, R, bytes, cudaMemcpyHostToDevice));
    if (L) {
        NK_CUDA(c, cudaMalloc(&c->defl_L, bytes));
        NK_CUDA(c, cudaMemcpy(c->defl_L, L, bytes, cudaMemcpyHostToDevice));
    } else {
        c->defl_L = c->defl_R;
    }
    std::vector<double> neg(m, -1.0), sg(m);
    double gap = 0.0;
    for (int i = 0; i < m; ++i) {
        const double re = lambda[2 * i], im = lambda[2 * i + 1];
        sg[i] = re > 0.0 ? 1.0 : (re < 0.0 ? -1.0 : 0.0);   // sgn(Re lambda), Eq. sgnz
        gap = std::max(gap, std::hypot(re, im));
    }
    NK_CUDA(c, cudaMalloc(&c->defl_neg, sizeof(double) * m));
    NK_CUDA(c, cudaMalloc(&c->defl_sgn, sizeof(double) * m));
    NK_CUDA(c, cudaMemcpy(c->defl_neg, neg.data(), sizeof(double) * m, cudaMemcpyHostToDevice));
    NK_CUDA(c, cudaMemcpy(c->defl_sgn, sg.data(), sizeof(double) * m, cudaMemcpyHostToDevice));
    c->defl_m = m;
    c->defl_gap = gap;
    return NK_OK;
}

// ---- eigensolver of the deflation (App. C step 1; Sec. 3) -------------------------
// k steps of the FP64 (two-sided) Lanczos recurrence from b with both bases
// kept, the eigenvalues of H_k by QL, the distinct ones nearest zero as
// candidates, their eigenvectors of H_k by inverse iteration lifted through
// the bases on the device, and the true residual of each.
int nk_eigs_smallest(nk_ctx* c, const double* b, int k, int m, double tol, double* lambda, double* R, double* L,
                     double* resid, int* found) {
    if (!c || !b || !lambda || !R || !found) return NK_EINVAL;
    *found = 0;
    if (int rb = busy(c)) return rb;
    if (m < 1 || m > NK_MAX_DEFL) return fail(c, NK_EINVAL, "need 1 <= m <= NK_MAX_DEFL");
    if (k < 2 * m + 2 || (k & 1)) return fail(c, NK_EINVAL, "k must be even and >= 2 m + 2");
    if (!(tol > 0.0)) return fail(c, NK_EINVAL, "tol must be positive");
    if (!c->links) return fail(c, NK_ESTATE, "no links loaded (nk_load_links)");
    if (!c->mu_set) return fail(c, NK_ESTATE, "mu and m_w not set (nk_set_mu_mw)");
    const bool ts = c->mu != 0.0;
    if (ts && !L) return fail(c, NK_EINVAL, "mu != 0: L receives the left eigenvectors");
    NK_CUDA(c, cudaSetDevice(c->device));
    cudaStream_t st = 0;
    const long N = c->N;
    const Geom g = geom_of(c);
    // the recurrence, FP64, with V_k and W_k kept
    const nk_launch lc = launch_cfg(c, 1, ts, false);
    Layout dry = carve(nullptr, g, 1, k, 2, ts, false, lc, false, Nesting(), true);
    int rc = ensure(c, c->ws, dry.total);
    if (rc) return rc;
    Layout Lw = carve((char*)c->ws.p, g, 1, k, 2, ts, false, lc, false, Nesting(), true);
    rc = ensure(c, c->staging, std::max(c->staging.bytes, sizeof(double2) * (size_t)N));
    if (rc) return rc;
    NK_CUDA(c, cudaMemcpy(c->staging.p, b, sizeof(double2) * (size_t)N, cudaMemcpyHostToDevice));
    NK_CUDA(c, cudaMemsetAsync(Lw.o.counters, 0, sizeof(unsigned), st));
    Launcher Lz;
    Lz.st = st;
    enqueue_load_sources(c, Lw.o, (const double*)c->staging.p, 1, Lz);
    enqueue_outer(c, Lw.o, schedule_of(c, NK_FP64, k), Lz);
    NK_CUDA(c, cudaGetLastError());
    std::vector<double2> al(k), be(k), ga(k);
    double xn = 0.0;
    int status = 0;
    NK_CUDA(c, cudaMemcpy(al.data(), Lw.o.alpha, sizeof(double2) * k, cudaMemcpyDeviceToHost));
    NK_CUDA(c, cudaMemcpy(be.data(), Lw.o.beta, sizeof(double2) * k, cudaMemcpyDeviceToHost));
    NK_CUDA(c, cudaMemcpy(ga.data(), Lw.o.gamma, sizeof(double2) * k, cudaMemcpyDeviceToHost));
    NK_CUDA(c, cudaMemcpy(&xn, Lw.o.xnorm, sizeof(double), cudaMemcpyDeviceToHost));
    NK_CUDA(c, cudaMemcpy(&status, Lw.o.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status == nk::kStatusZeroSource) return fail(c, NK_EINVAL, "zero start vector");
    if (status != nk::kStatusOK) return fail(c, NK_EBREAKDOWN, "Lanczos breakdown before step k");
    // H_k: diagonal H(j,j), sub-diagonal H(j+1,j) = beta_j, super-diagonal H(j,j+1) = gamma_j
    std::vector<nk::cplx> a(k), sub(k - 1), sup(k - 1);
    for (int j = 0; j < k; ++j) a[j] = ts ? nk::cplx(al[j].x, al[j].y) : nk::cplx(al[j].x, 0.0);
    for (int j = 0; j + 1 < k; ++j) {
        sub[j] = nk::cplx(be[j].x, ts ? be[j].y : 0.0);
        sup[j] = ts ? nk::cplx(ga[j].x, ga[j].y) : sub[j];
    }
    std::vector<nk::cplx> w;
    if (!nk::tridiag_eigvals(k, a.data(), sub.data(), sup.data(), w))
        return fail(c, NK_ENOTCONV, "QL iteration on H_k did not converge");
    // Clusters: the 2 m + 8 distinct eigenvalues of H_k nearest zero, each
    // with the number (up to kCopies) of its repeated values.  Floating-point
    // Lanczos repeats a converged eigenvalue, the copies agreeing to
    // rounding; the eigenvectors of H_k for the copies of one cluster are not
    // individually determined, only the invariant subspace they span is.
    std::vector<int> order(k);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int x, int y) { return std::abs(w[x]) < std::abs(w[y]); });
    constexpr int kCopies = 3;
    const int n_distinct = 2 * m + 8;
    auto same = [](nk::cplx x, nk::cplx y) { return std::abs(x - y) <= 1e-8 * std::max(1.0, std::abs(y)); };
    std::vector<nk::cplx> reps;
    std::vector<int> copies;
    for (int t = 0; t < k; ++t) {
        const nk::cplx v = w[order[t]];
        int q = 0;
        while (q < (int)reps.size() && !same(v, reps[q])) ++q;
        if (q == (int)reps.size()) {
            if (q == n_distinct) break;
            reps.push_back(v);
            copies.push_back(0);
        }
        copies[q] = std::min(copies[q] + 1, kCopies);
    }
    const int ncl = (int)reps.size();
    // Candidate Ritz vectors per cluster, as coefficients in the stored,
    // unnormalised bases: r = sum_j y_j q_j / n_j, l = sum_j z_j p_j / m_j
    // (n_0 = m_0 = |b|, n_{j+1} = beta_j, m_{j+1} = gamma_j^*).  For a cluster
    // of c copies: the c basis vectors of its invariant subspace (block
    // inverse iteration) and, for each pair of them, the combination whose
    // last component vanishes.  The residual of a Ritz vector V_k y is
    // |beta_k e_k^T y| |v_{k+1}| (A V_k = V_k H_k + beta_k v_{k+1} e_k^T), so
    // within the cluster's subspace that combination is the refined Ritz
    // vector, the one of least residual.  Left vectors the same way with
    // A^dagger W_k = W_k H_k^dagger + gamma_k^* w_{k+1} e_k^T.
    std::vector<int> owner_r, owner_l;
    std::vector<double2> coef_r, coef_l;
    auto add_candidates = [&](int q, bool left, std::vector<int>& owner, std::vector<double2>& coef) {
        std::vector<std::vector<nk::cplx>> Y;
        nk::tridiag_eigvecs(k, a.data(), sub.data(), sup.data(), reps[q], left, copies[q], Y);
        const int nb = (int)Y.size();
        for (int i = 0; i < nb; ++i)
            for (int j = i + 1; j < nb; ++j) {
                std::vector<nk::cplx> x(k);
                double nrm = 0.0;
                for (int t = 0; t < k; ++t) {
                    x[t] = Y[j][k - 1] * Y[i][t] - Y[i][k - 1] * Y[j][t];
                    nrm += std::norm(x[t]);
                }
                if (!(nrm > 0.0)) continue;
                for (nk::cplx& v : x) v /= std::sqrt(nrm);
                Y.push_back(x);
            }
        for (const auto& y : Y) {
            owner.push_back(q);
            for (int j = 0; j < k; ++j) {
                const nk::cplx nj = j == 0 ? nk::cplx(xn, 0.0) : (left ? std::conj(sup[j - 1]) : sub[j - 1]);
                const nk::cplx v = y[j] / nj;
                coef.push_back(make_double2(v.real(), v.imag()));
            }
        }
    };
    for (int q = 0; q < ncl; ++q) {
        add_candidates(q, false, owner_r, coef_r);
        if (ts) add_candidates(q, true, owner_l, coef_l);
    }
    // device: candidates in chunks of kChunk vectors, X = the lifted vectors,
    // AX = A X (A^dagger X for the left ones), residual |AX - theta X| / |X|
    constexpr int kChunk = 48;
    const int max_out = std::min(m, ncl);
    double2 *d_coef = nullptr, *d_X = nullptr, *d_AX = nullptr, *d_R = nullptr, *d_L = nullptr, *d_dot = nullptr,
            *d_abi = nullptr;
    auto release = [&] {
        for (double2* p : {d_coef, d_X, d_AX, d_R, d_L, d_dot, d_abi})
            if (p) cudaFree(p);
    };
    const size_t vb = sizeof(double2) * (size_t)N;
    if (cudaMalloc(&d_coef, sizeof(double2) * (size_t)kChunk * k) != cudaSuccess ||
        cudaMalloc(&d_X, vb * kChunk) != cudaSuccess || cudaMalloc(&d_AX, vb * kChunk) != cudaSuccess ||
        cudaMalloc(&d_R, vb * max_out) != cudaSuccess || (ts && cudaMalloc(&d_L, vb * max_out) != cudaSuccess) ||
        cudaMalloc(&d_dot, sizeof(double2) * 2 * kChunk) != cudaSuccess || cudaMalloc(&d_abi, vb) != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(c, NK_ENOMEM, "eigensolver buffers");
    }
#define NK_EIG_CUDA(x)                                              \
    do {                                                            \
        const cudaError_t e_ = (x);                                 \
        if (e_ != cudaSuccess) {                                    \
            release();                                              \
            return fail(c, NK_ECUDA, cudaGetErrorString(e_));       \
        }                                                           \
    } while (0)
    auto residuals = [&](const std::vector<double2>& coef, const std::vector<int>& owner, bool left,
                         std::vector<double>& res, std::vector<double>& nrm2) -> int {
        const int nc = (int)owner.size();
        res.assign(nc, 0.0);
        nrm2.assign(nc, 0.0);
        const double2* base = left ? nk::outer_p(Lw.o, 0, 0) : nk::outer_q(Lw.o, 0, 0);
        std::vector<double2> dd(kChunk), rr(kChunk);
        for (int t0 = 0; t0 < nc; t0 += kChunk) {
            const int n = std::min(kChunk, nc - t0);
            NK_EIG_CUDA(cudaMemcpy(d_coef, coef.data() + (size_t)t0 * k, sizeof(double2) * (size_t)n * k,
                                   cudaMemcpyHostToDevice));
            nk::launch_colcomb(base, N, k, d_coef, N, n, d_X, st);
            nk::DslashSet s0, s1;
            std::memset(&s0, 0, sizeof(s0));
            std::memset(&s1, 0, sizeof(s1));
            s0.in = d_X;
            s0.in_stride = N;
            s0.out = d_AX;
            s0.out_stride = N;
            s0.n = n;
            s0.dag = left ? 1 : 0;
            nk::launch_dslash(64, c->U64, g, s0, s1, kappa_of(c), c->mu, st);
            for (int g0 = 0; g0 < n; g0 += 12) {
                const int ng = std::min(12, n - g0);
                nk::VecCoefs ca, cb;
                for (int i = 0; i < ng; ++i) {
                    const nk::cplx th = reps[owner[t0 + g0 + i]];
                    const nk::cplx ths = left ? std::conj(th) : th;
                    ca.c[i] = make_double2(-ths.real(), -ths.imag());
                    cb.c[i] = make_double2(1.0, 0.0);
                }
                double2* ax = d_AX + (size_t)g0 * N;
                double2* x = d_X + (size_t)g0 * N;
                nk::launch_vlincomb(ax, x, N, ng, ca, cb, st);   // A x - theta x
                nk::launch_vdot(ax, ax, N, ng, d_dot, st);
                nk::launch_vdot(x, x, N, ng, d_dot + kChunk, st);
                NK_EIG_CUDA(cudaMemcpy(dd.data() + g0, d_dot, sizeof(double2) * ng, cudaMemcpyDeviceToHost));
                NK_EIG_CUDA(cudaMemcpy(rr.data() + g0, d_dot + kChunk, sizeof(double2) * ng, cudaMemcpyDeviceToHost));
            }
            for (int i = 0; i < n; ++i) {
                nrm2[t0 + i] = rr[i].x;
                res[t0 + i] = std::sqrt(dd[i].x / std::max(rr[i].x, 1e-300));
            }
        }
        return NK_OK;
    };
    std::vector<double> res_r, nrm_r, res_l, nrm_l;
    rc = residuals(coef_r, owner_r, false, res_r, nrm_r);
    if (rc) return rc;
    if (ts) {
        rc = residuals(coef_l, owner_l, true, res_l, nrm_l);
        if (rc) return rc;
    }
    // per cluster the right (and left) candidate of least residual; the
    // cluster's residual is the larger of the two
    std::vector<int> best_r(ncl, -1), best_l(ncl, -1);
    for (int t = 0; t < (int)owner_r.size(); ++t) {
        int& b_ = best_r[owner_r[t]];
        if (b_ < 0 || res_r[t] < res_r[b_]) b_ = t;
    }
    for (int t = 0; t < (int)owner_l.size(); ++t) {
        int& b_ = best_l[owner_l[t]];
        if (b_ < 0 || res_l[t] < res_l[b_]) b_ = t;
    }
    std::vector<double> res_cl(ncl);
    for (int q = 0; q < ncl; ++q) res_cl[q] = std::max(res_r[best_r[q]], ts ? res_l[best_l[q]] : 0.0);
    // the converged clusters (residual <= tol); of two whose eigenvalues lie
    // within their residuals of each other (approximations of one eigenvalue
    // of A) the one of smaller residual; the m nearest zero
    std::vector<int> keep;
    for (int q = 0; q < ncl; ++q) {
        if (!(res_cl[q] <= tol)) continue;
        int dup = -1;
        for (int i = 0; i < (int)keep.size(); ++i)
            if (std::abs(reps[q] - reps[keep[i]]) <= res_cl[q] + res_cl[keep[i]]) dup = i;
        if (dup < 0) keep.push_back(q);
        else if (res_cl[q] < res_cl[keep[dup]]) keep[dup] = q;
    }
    std::sort(keep.begin(), keep.end(), [&](int x, int y) { return std::abs(reps[x]) < std::abs(reps[y]); });
    if ((int)keep.size() > max_out) keep.resize(max_out);
    const int nf = (int)keep.size();
    // the chosen vectors, lifted again (the same coefficients and kernel give
    // the same vectors), normalised to |r| = 1 and <l, r> = 1
    for (int side = 0; side < (ts ? 2 : 1); ++side) {
        const std::vector<double2>& coef = side ? coef_l : coef_r;
        const std::vector<int>& best = side ? best_l : best_r;
        std::vector<double2> cc((size_t)nf * k);
        for (int i = 0; i < nf; ++i)
            std::copy(coef.begin() + (size_t)best[keep[i]] * k, coef.begin() + (size_t)(best[keep[i]] + 1) * k,
                      cc.begin() + (size_t)i * k);
        for (int t0 = 0; t0 < nf; t0 += kChunk) {
            const int n = std::min(kChunk, nf - t0);
            NK_EIG_CUDA(cudaMemcpy(d_coef, cc.data() + (size_t)t0 * k, sizeof(double2) * (size_t)n * k,
                                   cudaMemcpyHostToDevice));
            nk::launch_colcomb(side ? nk::outer_p(Lw.o, 0, 0) : nk::outer_q(Lw.o, 0, 0), N, k, d_coef, N, n,
                               (side ? d_L : d_R) + (size_t)t0 * N, st);
        }
    }
    for (int g0 = 0; g0 < nf; g0 += 12) {
        const int ng = std::min(12, nf - g0);
        nk::VecCoefs ca, cb;
        for (int i = 0; i < ng; ++i) {
            ca.c[i] = make_double2(0.0, 0.0);
            cb.c[i] = make_double2(1.0 / std::sqrt(nrm_r[best_r[keep[g0 + i]]]), 0.0);
        }
        double2* rg = d_R + (size_t)g0 * N;
        nk::launch_vlincomb(rg, rg, N, ng, ca, cb, st);   // |r| = 1
        if (ts) {
            double2* lg = d_L + (size_t)g0 * N;
            std::vector<double2> s(ng);
            nk::launch_vdot(lg, rg, N, ng, d_dot, st);
            NK_EIG_CUDA(cudaMemcpy(s.data(), d_dot, sizeof(double2) * ng, cudaMemcpyDeviceToHost));
            for (int i = 0; i < ng; ++i) {
                const nk::cplx sc = 1.0 / std::conj(nk::cplx(s[i].x, s[i].y));   // l <- l / <l, r>^*
                cb.c[i] = make_double2(sc.real(), sc.imag());
            }
            nk::launch_vlincomb(lg, lg, N, ng, ca, cb, st);
        }
    }
    // The Rayleigh quotient of each returned pair, theta' = <l, A r> (<l, r> =
    // 1; Hermitian: <r, A r>, |r| = 1), with its residuals: H_k's eigenvalue
    // is good to about the residual, theta' to about the product of the left
    // and right residuals.  theta' replaces it where its residual is not
    // larger (the Hermitian quotient minimises |A r - theta r|; the two-sided
    // one need not).
    std::vector<nk::cplx> th_out(nf);
    std::vector<double> res_out(nf);
    {
        std::vector<double2> dd(12), rr(12);
        for (int t0 = 0; t0 < nf; t0 += kChunk) {
            const int n = std::min(kChunk, nf - t0);
            for (int side = 0; side < (ts ? 2 : 1); ++side) {
                double2* v = (side ? d_L : d_R) + (size_t)t0 * N;
                double2* av = side ? d_AX : d_X;
                nk::DslashSet s0, s1;
                std::memset(&s0, 0, sizeof(s0));
                std::memset(&s1, 0, sizeof(s1));
                s0.in = v;
                s0.in_stride = N;
                s0.out = av;
                s0.out_stride = N;
                s0.n = n;
                s0.dag = side;
                nk::launch_dslash(64, c->U64, g, s0, s1, kappa_of(c), c->mu, st);
                for (int g0 = 0; g0 < n; g0 += 12) {
                    const int ng = std::min(12, n - g0);
                    if (side == 0) {   // theta' = <l, A r>
                        nk::launch_vdot((ts ? d_L : d_R) + (size_t)(t0 + g0) * N, av + (size_t)g0 * N, N, ng, d_dot,
                                        st);
                        NK_EIG_CUDA(cudaMemcpy(dd.data(), d_dot, sizeof(double2) * ng, cudaMemcpyDeviceToHost));
                        for (int i = 0; i < ng; ++i)
                            th_out[t0 + g0 + i] = nk::cplx(dd[i].x, ts ? dd[i].y : 0.0);
                    }
                    nk::VecCoefs ca, cb;
                    for (int i = 0; i < ng; ++i) {
                        const nk::cplx t = side ? std::conj(th_out[t0 + g0 + i]) : th_out[t0 + g0 + i];
                        ca.c[i] = make_double2(-t.real(), -t.imag());
                        cb.c[i] = make_double2(1.0, 0.0);
                    }
                    double2* ag = av + (size_t)g0 * N;
                    double2* vg = v + (size_t)g0 * N;
                    nk::launch_vlincomb(ag, vg, N, ng, ca, cb, st);   // A v - theta v
                    nk::launch_vdot(ag, ag, N, ng, d_dot, st);
                    nk::launch_vdot(vg, vg, N, ng, d_dot + kChunk, st);
                    NK_EIG_CUDA(cudaMemcpy(dd.data(), d_dot, sizeof(double2) * ng, cudaMemcpyDeviceToHost));
                    NK_EIG_CUDA(cudaMemcpy(rr.data(), d_dot + kChunk, sizeof(double2) * ng, cudaMemcpyDeviceToHost));
                    for (int i = 0; i < ng; ++i) {
                        const double r_ = std::sqrt(dd[i].x / std::max(rr[i].x, 1e-300));
                        double& ro = res_out[t0 + g0 + i];
                        ro = side ? std::max(ro, r_) : r_;
                    }
                }
            }
        }
    }
    for (int i = 0; i < nf; ++i) {
        const int q = keep[i];
        const bool refined = res_out[i] <= res_cl[q];
        const nk::cplx lam = refined ? th_out[i] : reps[q];
        nk::launch_soa_to_abi(d_R + (size_t)i * N, N, d_abi, N, nullptr, 0, c->V, 1, st);
        NK_EIG_CUDA(cudaMemcpy(R + (size_t)i * 2 * N, d_abi, vb, cudaMemcpyDeviceToHost));
        if (ts) {
            nk::launch_soa_to_abi(d_L + (size_t)i * N, N, d_abi, N, nullptr, 0, c->V, 1, st);
            NK_EIG_CUDA(cudaMemcpy(L + (size_t)i * 2 * N, d_abi, vb, cudaMemcpyDeviceToHost));
        } else if (L) {
            std::memcpy(L + (size_t)i * 2 * N, R + (size_t)i * 2 * N, vb);
        }
        lambda[2 * i] = lam.real();
        lambda[2 * i + 1] = ts ? lam.imag() : 0.0;
        if (resid) resid[i] = refined ? res_out[i] : res_cl[q];
    }
    NK_EIG_CUDA(cudaGetLastError());
#undef NK_EIG_CUDA
    release();
    *found = nf;
    if (nf < m) return fail(c, NK_ENOTCONV, "fewer than m eigenpairs reached tol at this k");
    return NK_OK;
}

int nk_set_nesting(nk_ctx* c, int n_deeper, const int* ells) {
    if (!c) return NK_EINVAL;
    if (n_deeper < 0 || n_deeper > NK_MAX_LEVELS - 1 || (n_deeper > 0 && !ells))
        return fail(c, NK_EINVAL, "n_deeper must be in [0, NK_MAX_LEVELS - 1] with its sizes");
    for (int i = 0; i < n_deeper; ++i)
        if (ells[i] < 2 || (ells[i] & 1) || (i > 0 && ells[i] > ells[i - 1]))
            return fail(c, NK_EINVAL, "level sizes must be even, >= 2 and non-increasing");
    c->nest.n = n_deeper;
    for (int i = 0; i < NK_MAX_LEVELS - 1; ++i) c->nest.ell[i] = i < n_deeper ? ells[i] : 0;
    return NK_OK;
}

int nk_set_adapt_start(nk_ctx* c, int k_first) {
    if (!c || k_first < 0) return NK_EINVAL;
    c->adapt_start = k_first;
    return NK_OK;
}

static void clear_graphs(nk_ctx* c) {
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.second.first);
    c->graphs.clear();
}

static int shape_args(nk_ctx* c, int n_rhs) {
    if (!c) return NK_EINVAL;
    if (n_rhs < 1 || n_rhs > NK_MAX_RHS) return fail(c, NK_EINVAL, "bad n_rhs");
    if (!c->mu_set) return fail(c, NK_ESTATE, "(mu, m_w) not set: the launch shape depends on mu != 0");
    return NK_OK;
}

int nk_set_launch(nk_ctx* c, int n_rhs, unsigned flags, const nk_launch* l) {
    int rc = shape_args(c, n_rhs);
    if (rc) return rc;
    if (!l || !valid_launch(*l)) return fail(c, NK_EINVAL, "bad launch shape");
    c->tune[std::make_tuple(n_rhs, c->mu != 0.0 ? 1 : 0, (flags & NK_MIXED) ? 1 : 0)] = *l;
    clear_graphs(c);
    return NK_OK;
}

int nk_get_launch(nk_ctx* c, int n_rhs, unsigned flags, nk_launch* l) {
    int rc = shape_args(c, n_rhs);
    if (rc) return rc;
    if (!l) return fail(c, NK_EINVAL, "null pointer");
    *l = launch_cfg(c, n_rhs, c->mu != 0.0, (flags & NK_MIXED) != 0);
    return NK_OK;
}

// Autotuner timing: the outer recurrence is run for kTuneWarm steps from the
// synthetic source in `src` with launch shape lc, then the two kernels of
// step kTuneWarm -- the fused stencil in precision `prec` (32, 48 or 64) and
// step 2 -- are launched kTuneReps times in turn and timed with CUDA events
// (the minimum over kTuneRounds rounds, per step).  Alternating the two keeps the
// dependency between them that a solve has (timing one kernel alone lets
// consecutive launches overlap and favours other shapes); repeating a step
// recomputes it (step 2 subtracts once more), which leaves the timing
// representative.  Step 2 skips the copy for the next stencil there (the next
// repetition's stencil must read q_j again), a small part of its traffic.
constexpr int kTuneWarm = 8, kTuneReps = 50, kTuneRounds = 3;
static int time_kernel(nk_ctx* c, const double* src, int n_rhs, bool mixed, int prec, const nk_launch& lc,
                       cudaStream_t st, float* per_launch_ms) {
    const bool ts = c->mu != 0.0;
    const int k = 2 * kTuneWarm;
    Layout dry = carve(nullptr, geom_of(c), n_rhs, k, 2, ts, false, lc, mixed);
    int rc = ensure(c, c->ws, dry.total);
    if (rc) return rc;
    Layout Lw = carve((char*)c->ws.p, geom_of(c), n_rhs, k, 2, ts, false, lc, mixed);
    NK_CUDA(c, cudaMemsetAsync(Lw.o.counters, 0, sizeof(unsigned) * n_rhs, st));
    Launcher L;
    L.st = st;
    enqueue_load_sources(c, Lw.o, src, n_rhs, L);
    // the copies of the stencil input that `prec` reads are made by the last warm step
    Schedule sch;
    sch.mixed = mixed;
    sch.j0 = prec == 48 ? k : 0;
    // the epilogue the solves will use: the two-float recurrence where it is
    // selected (nk_set_df_recurrence; for the two-float stencil only from step 0),
    // else FP64
    if (mixed) Lw.o.ring_from = (prec == 48 ? c->j1 == 0 : c->j1 >= 0) ? 0 : k;
    const bool ring = mixed && Lw.o.ring_from == 0;
    enqueue_outer(c, Lw.o, sch, L, kTuneWarm);
    const Geom g = geom_of(c);
    const void* U = prec == 64 ? (const void*)c->U64 : (prec == 48 ? (const void*)c->Udf : (const void*)c->U32);
    EventPair ev;   // destroyed on every return
    NK_CUDA(c, cudaEventCreate(&ev.e0));
    NK_CUDA(c, cudaEventCreate(&ev.e1));
    const cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    float best = 1e30f;
    for (int round = 0; round < kTuneRounds; ++round) {
        NK_CUDA(c, cudaEventRecord(e0, st));
        for (int r = 0; r < kTuneReps; ++r) {
            nk::launch_dslash_step1(prec, U, g, Lw.o, kTuneWarm, kappa_of(c), c->mu, st);
            // no copy for the next stencil: the stencil of the next repetition
            // must read q_j again, so that every repetition recomputes the same step
            nk::launch_outer_step2(Lw.o, kTuneWarm, nk::kCopyNone, ring, false, st);
        }
        NK_CUDA(c, cudaEventRecord(e1, st));
        NK_CUDA(c, cudaGetLastError());
        NK_CUDA(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        NK_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms / kTuneReps);
    }
    *per_launch_ms = best;
    return NK_OK;
}

int nk_autotune(nk_ctx* c, int n_rhs, unsigned flags, const char* cache_path, nk_launch* out, double* ms_per_step) {
    int rc = shape_args(c, n_rhs);
    if (rc) return rc;
    if ((rc = busy(c))) return rc;
    if (!c->links) return fail(c, NK_ESTATE, "links not loaded");
    NK_CUDA(c, cudaSetDevice(c->device));
    const int ts = c->mu != 0.0 ? 1 : 0;
    const int mixed = (flags & NK_MIXED) ? 1 : 0;
    if (cache_path) {
        if (FILE* f = std::fopen(cache_path, "r")) {
            char tag[32];
            int d[4], nr, t2, mx, th, od, bl, eth, eod, sp, esp;
            double ms;
            bool found = false;
            nk_launch hit;
            while (std::fscanf(f, "%31s %d %d %d %d %d %d %d %d %d %d %d %d %d %d %lf", tag, &d[0], &d[1], &d[2],
                               &d[3], &nr, &t2, &mx, &th, &od, &bl, &eth, &eod, &sp, &esp, &ms) == 16) {
                if (std::strcmp(tag, "nk_launch") != 0) break;
                if (d[0] == c->dims[0] && d[1] == c->dims[1] && d[2] == c->dims[2] && d[3] == c->dims[3] &&
                    nr == n_rhs && t2 == ts && mx == mixed) {
                    hit.stencil_threads = th;
                    hit.stencil_order = od;
                    hit.step2_blocks = bl;
                    hit.early_threads = eth;
                    hit.early_order = eod;
                    hit.stencil_split = sp;
                    hit.early_split = esp;
                    if (valid_launch(hit)) {
                        found = true;
                        if (ms_per_step) *ms_per_step = ms;
                    }
                }
            }
            std::fclose(f);
            if (found) {
                c->tune[std::make_tuple(n_rhs, ts, mixed)] = hit;
                clear_graphs(c);
                if (out) *out = hit;
                return NK_OK;
            }
        }
    }
    // synthetic source: every component 0x3F3F3F3F3F3F3F3F (about 4.8e-4)
    const size_t sb = sizeof(double2) * (size_t)c->N * n_rhs;
    rc = ensure(c, c->staging, std::max(sb, c->staging.bytes));
    if (rc) return rc;
    cudaStream_t st;
    NK_CUDA(c, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    const cudaError_t e_fill = cudaMemsetAsync(c->staging.p, 0x3F, sb, st);
    if (e_fill != cudaSuccess) {
        cudaStreamDestroy(st);
        return cuda_fail(c, e_fill, "autotune input");
    }
    const double* src = (const double*)c->staging.p;
    nk_launch best = launch_cfg(c, n_rhs, ts != 0, mixed != 0);
    best.stencil_threads = 128;
    best.stencil_order = 0;
    best.early_threads = 128;
    best.early_order = 0;
    best.stencil_split = 1;
    best.early_split = 1;
    const int b0 = blocks_per_rhs(c->N, n_rhs);
    best.step2_blocks = b0;
    // each kernel of an outer step is tuned on its own
    auto fail_out = [&](int code) { cudaStreamDestroy(st); return code; };
    float t_st = 1e30f, t_early = 1e30f, t_s2 = 1e30f;
    nk_launch cand = best;
    for (int th : {64, 128, 256})
        for (int od : {0, 1})
            for (int sp : {1, 3}) {
                float t;
                if (!mixed) {
                    // the FP32 stencil of the mixed schedule has one shape (stencil32.cu);
                    // the FP64 stencil of NK_FP64 is tuned
                    nk_launch l = best;
                    l.stencil_threads = th;
                    l.stencil_order = od;
                    l.stencil_split = sp;
                    rc = time_kernel(c, src, n_rhs, false, 64, l, st, &t);
                    if (rc) return fail_out(rc);
                    if (t < t_st) { t_st = t; cand.stencil_threads = th; cand.stencil_order = od; cand.stencil_split = sp; }
                } else {
                    nk_launch e = best;
                    e.early_threads = th;
                    e.early_order = od;
                    e.early_split = sp;
                    rc = time_kernel(c, src, n_rhs, true, 48, e, st, &t);
                    if (rc) return fail_out(rc);
                    if (t < t_early) { t_early = t; cand.early_threads = th; cand.early_order = od; cand.early_split = sp; }
                }
            }
    for (int bl : {std::max(1, b0 / 2), b0, 2 * b0, 4 * b0, 8 * b0}) {
        nk_launch l = best;
        l.stencil_threads = cand.stencil_threads;
        l.stencil_order = cand.stencil_order;
        l.stencil_split = cand.stencil_split;
        l.step2_blocks = std::min(bl, 4096);
        float t;
        rc = time_kernel(c, src, n_rhs, mixed != 0, mixed ? 32 : 64, l, st, &t);
        if (rc) return fail_out(rc);
        if (t < t_s2) { t_s2 = t; cand.step2_blocks = l.step2_blocks; }
    }
    best = cand;
    // reported: the time of one outer step after j0 (stencil + step 2)
    const float t_best = t_s2;
    cudaStreamDestroy(st);
    c->tune[std::make_tuple(n_rhs, ts, mixed)] = best;
    clear_graphs(c);
    const double per_step = t_best;
    if (out) *out = best;
    if (ms_per_step) *ms_per_step = per_step;
    if (cache_path) {
        if (FILE* f = std::fopen(cache_path, "a")) {
            std::fprintf(f, "nk_launch %d %d %d %d %d %d %d %d %d %d %d %d %d %d %.17g\n", c->dims[0], c->dims[1],
                         c->dims[2], c->dims[3], n_rhs, ts, mixed, best.stencil_threads, best.stencil_order,
                         best.step2_blocks, best.early_threads, best.early_order, best.stencil_split,
                         best.early_split, per_step);
            std::fclose(f);
        } else {
            return fail(c, NK_EINVAL, "cannot append to the tuning cache file");
        }
    }
    return NK_OK;
}

int nk_sign_apply_dev(nk_ctx* c, const double* b_dev, int n_rhs, int k, int ell, double tol, double p,
                      unsigned flags, double* y_dev, nk_stats* st, void* stream) {
    if (!c || !b_dev || !y_dev) return NK_EINVAL;
    return solve_dev(c, b_dev, n_rhs, k, ell, tol, p, flags, y_dev, st, (cudaStream_t)stream, false);
}

static int host_solve(nk_ctx* c, const double* b, int n_rhs, int k, int ell, double tol, double p,
                      unsigned flags, double* y, nk_stats* st, bool overlap) {
    if (!c || !b || !y) return NK_EINVAL;
    int rc = check_solve_args(c, n_rhs, k, ell, tol);
    if (rc) return rc;
    NK_CUDA(c, cudaSetDevice(c->device));
    const size_t bytes = sizeof(double2) * (size_t)c->N * n_rhs;
    rc = ensure(c, c->staging, 2 * NK_MAX_RHS * sizeof(double2) * (size_t)c->N);
    if (rc) return rc;
    double* bd = (double*)c->staging.p;
    double* yd = bd + 2 * (size_t)c->N * NK_MAX_RHS;
    NK_CUDA(c, cudaMemcpy(bd, b, bytes, cudaMemcpyHostToDevice));
    rc = solve_dev(c, bd, n_rhs, k, ell, tol, p, flags, yd, st, 0, overlap);
    if (rc != NK_OK && rc != NK_EBREAKDOWN && rc != NK_ERHI && rc != NK_ENOTCONV) return rc;
    cudaError_t e = cudaMemcpy(y, yd, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy y");
    return rc;
}

int nk_sign_apply(nk_ctx* c, const double* b, int n_rhs, int k, int ell, double tol, double p,
                  unsigned flags, double* y, nk_stats* st) {
    return host_solve(c, b, n_rhs, k, ell, tol, p, flags, y, st, false);
}

int nk_overlap_apply(nk_ctx* c, const double* b, int n_rhs, int k, int ell, double tol, unsigned flags,
                     double* y, nk_stats* st) {
    return host_solve(c, b, n_rhs, k, ell, tol, 0.0, flags, y, st, true);
}

int nk_overlap_apply_dev(nk_ctx* c, const double* b_dev, int n_rhs, int k, int ell, double tol,
                         unsigned flags, double* y_dev, nk_stats* st, void* stream) {
    if (!c || !b_dev || !y_dev) return NK_EINVAL;
    return solve_dev(c, b_dev, n_rhs, k, ell, tol, 0.0, flags, y_dev, st, (cudaStream_t)stream, true);
}

int nk_stencil32_dev(nk_ctx* c, const float* in_dev, float* out_dev, int n_rhs, void* stream) {
    if (!c) return NK_EINVAL;
    if (!in_dev || !out_dev) return fail(c, NK_EINVAL, "null pointer");
    if ((reinterpret_cast<uintptr_t>(in_dev) & 15) || (reinterpret_cast<uintptr_t>(out_dev) & 15))
        return fail(c, NK_EINVAL, "in_dev and out_dev must be 16-byte aligned");
    if (n_rhs < 1 || n_rhs > NK_MAX_RHS) return fail(c, NK_EINVAL, "n_rhs must be in [1, 12]");
    if (!c->links) return fail(c, NK_ESTATE, "no links loaded");
    if (!c->mu_set) return fail(c, NK_ESTATE, "mu and m_w not set");
    NK_CUDA(c, cudaSetDevice(c->device));
    const long vs = c->N / 2;   // float4 per vector
    nk::Stencil32Set s;
    s.in_a = reinterpret_cast<const float4*>(in_dev);
    s.in_d = s.in_a + (size_t)n_rhs * vs;
    s.out_a = reinterpret_cast<float4*>(out_dev);
    s.out_d = s.out_a + (size_t)n_rhs * vs;
    s.vstride = vs;
    s.n_a = s.n_d = n_rhs;
    s.scale = nullptr;
    nk::launch_stencil32(c->U32, geom_of(c), s, kappa_of(c), c->mu, (cudaStream_t)stream);
    NK_CUDA(c, cudaGetLastError());
    return NK_OK;
}

int nk_dslash_dev(nk_ctx* c, const double* in_dev, double* out_dev, int n_vec, int dagger, int precision,
                  void* stream) {
    if (!c || !in_dev || !out_dev || n_vec < 1 || n_vec > 2 * NK_MAX_RHS) return NK_EINVAL;
    if (precision != 32 && precision != 48 && precision != 64)
        return fail(c, NK_EINVAL, "precision must be 32, 48 or 64");
    if (!c->links) return fail(c, NK_ESTATE, "no links loaded");
    if (!c->mu_set) return fail(c, NK_ESTATE, "mu and m_w not set");
    NK_CUDA(c, cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    const long N = c->N;
    if (precision == 32) {
        // FP32: the multi-RHS stencil on FP32 pair-layout copies (input rounded once)
        const size_t vb = align_up(sizeof(float2) * N * n_vec);
        int rc = ensure(c, c->staging, std::max(2 * vb, c->staging.bytes));
        if (rc) return rc;
        float4* in32 = (float4*)c->staging.p;
        float4* out32 = (float4*)((char*)c->staging.p + vb);
        nk::launch_abi_to_f32pair((const double2*)in_dev, N, in32, N / 2, c->V, n_vec, st);
        nk::Stencil32Set s;
        s.in_a = s.in_d = in32;
        s.out_a = s.out_d = out32;
        s.vstride = N / 2;
        s.n_a = dagger ? 0 : n_vec;
        s.n_d = dagger ? n_vec : 0;
        s.scale = nullptr;
        nk::launch_stencil32(c->U32, geom_of(c), s, kappa_of(c), c->mu, st);
        nk::launch_f32pair_to_abi(out32, N / 2, (double2*)out_dev, N, c->V, n_vec, st);
        NK_CUDA(c, cudaGetLastError());
        return NK_OK;
    }
    // scratch: SoA input (FP64 or two-float) and SoA output
    size_t bytes = align_up(sizeof(double2) * N * n_vec) * 3;
    int rc = ensure(c, c->staging, std::max(bytes, c->staging.bytes));
    if (rc) return rc;
    double2* in_soa = (double2*)c->staging.p;
    double2* out_soa = (double2*)((char*)c->staging.p + align_up(sizeof(double2) * N * n_vec));
    float2* in32 = (float2*)((char*)out_soa + align_up(sizeof(double2) * N * n_vec));
    nk::launch_abi_to_soa((const double2*)in_dev, N, in_soa, N, c->V, n_vec, st);
    if (precision == 48) {
        // the multi-RHS two-float stencil of the solver's early steps
        nk::launch_to_df(in_soa, N, (nk::dfc*)in32, N, N, n_vec, st);
        nk::StencilDfSet sd;
        sd.in_a = sd.in_d = (const nk::dfc*)in32;
        sd.in_stride = N;
        sd.out_a = sd.out_d = out_soa;
        sd.out_stride = N;
        sd.n_a = dagger ? 0 : n_vec;
        sd.n_d = dagger ? n_vec : 0;
        sd.scale = nullptr;
        nk::launch_stencil_df(c->Udf, geom_of(c), sd, kappa_of(c), c->mu, st);
        nk::launch_soa_to_abi(out_soa, N, (double2*)out_dev, N, nullptr, 0, c->V, n_vec, st);
        NK_CUDA(c, cudaGetLastError());
        return NK_OK;
    }
    nk::DslashSet s0, s1;
    std::memset(&s0, 0, sizeof(s0));
    std::memset(&s1, 0, sizeof(s1));
    s0.in = in_soa;
    s0.in_stride = N;
    s0.out = out_soa;
    s0.out_stride = N;
    s0.n = n_vec;
    s0.dag = dagger ? 1 : 0;
    nk::launch_dslash(precision, precision == 48 ? (const void*)c->Udf : (const void*)c->U64, geom_of(c), s0, s1,
                      kappa_of(c), c->mu, st);
    nk::launch_soa_to_abi(out_soa, N, (double2*)out_dev, N, nullptr, 0, c->V, n_vec, st);
    NK_CUDA(c, cudaGetLastError());
    return NK_OK;
}

int nk_outer_lanczos_dev(nk_ctx* c, const double* b_dev, int n_rhs, int k, unsigned flags, double* alpha,
                         double* beta, double* gamma, double* xnorm, void* stream) {
    int rc = check_solve_args(c, n_rhs, k, 2, 0.0);
    if (rc) return rc;
    if (!b_dev || !alpha || !beta || !gamma || !xnorm) return fail(c, NK_EINVAL, "null pointer");
    NK_CUDA(c, cudaSetDevice(c->device));
    cudaStream_t st = (cudaStream_t)stream;
    const bool ts = c->mu != 0.0;
    const nk_launch lc = launch_cfg(c, n_rhs, ts, (flags & NK_MIXED) != 0);
    const bool mixed = (flags & NK_MIXED) != 0;
    Layout dry = carve(nullptr, geom_of(c), n_rhs, k, 2, ts, false, lc, mixed);
    rc = ensure(c, c->ws, dry.total);
    if (rc) return rc;
    Layout Lw = carve((char*)c->ws.p, geom_of(c), n_rhs, k, 2, ts, false, lc, mixed);
    NK_CUDA(c, cudaMemsetAsync(Lw.o.counters, 0, sizeof(unsigned) * n_rhs, st));
    Launcher L;
    L.st = st;
    enqueue_load_sources(c, Lw.o, b_dev, n_rhs, L);
    if (mixed) Lw.o.ring_from = effective_j1(c);
    enqueue_outer(c, Lw.o, schedule_of(c, flags, k), L);
    NK_CUDA(c, cudaGetLastError());
    const size_t cb = sizeof(double2) * (size_t)k * n_rhs;
    NK_CUDA(c, cudaMemcpyAsync(alpha, Lw.o.alpha, cb, cudaMemcpyDeviceToHost, st));
    NK_CUDA(c, cudaMemcpyAsync(beta, Lw.o.beta, cb, cudaMemcpyDeviceToHost, st));
    NK_CUDA(c, cudaMemcpyAsync(gamma, Lw.o.gamma, cb, cudaMemcpyDeviceToHost, st));
    NK_CUDA(c, cudaMemcpyAsync(xnorm, Lw.o.xnorm, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost, st));
    std::vector<int> status(n_rhs);
    NK_CUDA(c, cudaMemcpyAsync(status.data(), Lw.o.status, sizeof(int) * n_rhs, cudaMemcpyDeviceToHost, st));
    NK_CUDA(c, cudaStreamSynchronize(st));
    for (int r = 0; r < n_rhs; ++r)
        if (status[r] == nk::kStatusBreakdown)
            return fail(c, NK_EBREAKDOWN, "two-sided Lanczos: serious breakdown (delta = 0)");
    return NK_OK;
}

int nk_inner_sign(nk_ctx* c, const double* alpha, const double* beta, const double* gamma, int n_rhs, int k,
                  int ell, double p, int hermitian, double* cout, nk_stats* st) {
    if (!c || !alpha || !beta || !gamma || !cout) return NK_EINVAL;
    if (int rb = busy(c)) return rb;
    if (n_rhs < 1 || n_rhs > NK_MAX_RHS || k < 2 || ell < 2 || ell > k || ell > 256 || (k & 1) || (ell & 1) ||
        k > nk::kMaxInnerK)
        return fail(c, NK_EINVAL, "bad n_rhs, k or l");
    NK_CUDA(c, cudaSetDevice(c->device));
    const bool ts = hermitian == 0;
    Geom tiny;
    tiny.Lx = tiny.Ly = tiny.Lz = tiny.Lt = 1;
    tiny.V = 1;
    tiny.antiperiodic = 0;
    nk_launch one;
    one.stencil_threads = 64;
    one.stencil_order = 0;
    one.step2_blocks = 1;
    one.early_threads = 64;
    one.early_order = 0;
    one.stencil_split = 1;
    one.early_split = 1;
    Layout dry = carve(nullptr, tiny, n_rhs, k, ell, ts, true, one, false, c->nest);
    int rc = ensure(c, c->inner_tmp, std::max(dry.total, c->inner_tmp.bytes));
    if (rc) return rc;
    Layout Lw = carve((char*)c->inner_tmp.p, tiny, n_rhs, k, ell, ts, true, one, false, c->nest);
    const size_t cb = sizeof(double2) * (size_t)k * n_rhs;
    NK_CUDA(c, cudaMemcpy(Lw.o.alpha, alpha, cb, cudaMemcpyHostToDevice));
    NK_CUDA(c, cudaMemcpy(Lw.o.beta, beta, cb, cudaMemcpyHostToDevice));
    NK_CUDA(c, cudaMemcpy(Lw.o.gamma, gamma, cb, cudaMemcpyHostToDevice));
    NK_CUDA(c, cudaMemset(Lw.o.status, 0, sizeof(int) * n_rhs));
    nk::Inner in = Lw.in;
    in.p_fixed = p > 0.0 ? p : 0.0;
    in.p_shared = p < 0.0 ? 1 : 0;
    Launcher L;
    L.st = 0;
    const int* iters_dev = in.rhi_iters;
    cudaError_t e = enqueue_inner_chain(Lw, in, L, &iters_dev);
    if (e != cudaSuccess) return cuda_fail(c, e, "launch_rhi");
    nk::launch_inner_combine(in, 0);
    NK_CUDA(c, cudaGetLastError());
    NK_CUDA(c, cudaDeviceSynchronize());
    NK_CUDA(c, cudaMemcpy(cout, in.c, cb, cudaMemcpyDeviceToHost));
    std::vector<int> status(n_rhs), iters(n_rhs);
    std::vector<double> pv(n_rhs), zmin(n_rhs), zmax(n_rhs);
    NK_CUDA(c, cudaMemcpy(status.data(), in.status, sizeof(int) * n_rhs, cudaMemcpyDeviceToHost));
    NK_CUDA(c, cudaMemcpy(iters.data(), iters_dev, sizeof(int) * n_rhs, cudaMemcpyDeviceToHost));
    NK_CUDA(c, cudaMemcpy(pv.data(), in.p, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost));
    NK_CUDA(c, cudaMemcpy(zmin.data(), in.zmin, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost));
    NK_CUDA(c, cudaMemcpy(zmax.data(), in.zmax, sizeof(double) * n_rhs, cudaMemcpyDeviceToHost));
    int worst = NK_OK;
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->n_rhs = n_rhs;
        st->k_used = k;
        st->ell_used = ell;
    }
    for (int r = 0; r < n_rhs; ++r) {
        int code = status_to_code(status[r]);
        if (code != NK_OK && worst == NK_OK) worst = code;
        if (st) {
            st->rhi_iters[r] = iters[r];
            st->status[r] = code;
            st->p[r] = pv[r];
            st->z_min[r] = zmin[r];
            st->z_max[r] = zmax[r];
        }
    }
    if (worst != NK_OK) return fail(c, worst, "inner sign failed (breakdown, singular p H_k or RHi)");
    return NK_OK;
}

int nk_features(nk_ctx* c, const double* b_dev, float* features, void* stream) {
    if (!c || !b_dev || !features) return c ? fail(c, NK_EINVAL, "null pointer") : NK_EINVAL;
    if (int rb = busy(c)) return rb;
    if (!c->links || !c->mu_set) return fail(c, NK_ESTATE, "links or (mu, m_w) not set");
    const int k = 32, ell = 32;
    std::vector<double> al(2 * k), be(2 * k), ga(2 * k), cf(2 * k);
    double xn = 0.0;
    int rc = nk_outer_lanczos_dev(c, b_dev, 1, k, NK_FP64, al.data(), be.data(), ga.data(), &xn, stream);
    if (rc) return rc;
    if (!(xn > 0.0)) return fail(c, NK_EINVAL, "zero source");
    nk_stats ist;
    rc = nk_inner_sign(c, al.data(), be.data(), ga.data(), 1, k, ell, 0.0, c->mu == 0.0 ? 1 : 0, cf.data(), &ist);
    if (rc) return rc;

    // mean plaquette: per-block partial sums, summed here in a fixed order
    const Geom g = geom_of(c);
    const int nb = nk::plaquette_blocks(g);
    rc = ensure(c, c->inner_tmp, std::max(c->inner_tmp.bytes, sizeof(double) * (size_t)nb));
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    nk::launch_plaquette(c->U64, g, (double*)c->inner_tmp.p, st);
    NK_CUDA(c, cudaGetLastError());
    std::vector<double> part(nb);
    NK_CUDA(c, cudaMemcpyAsync(part.data(), c->inner_tmp.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    NK_CUDA(c, cudaStreamSynchronize(st));
    double plaq = 0.0;
    for (int i = 0; i < nb; ++i) plaq += part[i];
    plaq /= 6.0 * c->V;

    double f[NK_MLP_IN];
    f[0] = c->mu;
    f[1] = c->m_w;
    f[2] = std::log10((double)c->V);
    f[3] = plaq;
    f[4] = std::log10(ist.z_min[0]);
    f[5] = std::log10(ist.z_max[0]);
    f[6] = f[5] - f[4];
    f[7] = std::log10(ist.p[0]);
    double m = 0, s2 = 0, im = 0;
    for (int j = 0; j < k; ++j) {
        m += al[2 * j];
        im = std::max(im, std::fabs(al[2 * j + 1]));
    }
    m /= k;
    for (int j = 0; j < k; ++j) s2 += (al[2 * j] - m) * (al[2 * j] - m);
    f[8] = m;
    f[9] = std::sqrt(s2 / k);
    f[10] = im;
    const int nsub = k - 1;
    double bm = 0, bs = 0, sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (int j = 0; j < nsub; ++j) {
        const double a = std::hypot(be[2 * j], be[2 * j + 1]);
        const double ly = std::log(std::max(a, 1e-300));
        bm += a;
        sx += j; sy += ly; sxx += (double)j * j; sxy += j * ly;
    }
    bm /= nsub;
    for (int j = 0; j < nsub; ++j) {
        const double a = std::hypot(be[2 * j], be[2 * j + 1]);
        bs += (a - bm) * (a - bm);
    }
    f[11] = bm;
    f[12] = std::sqrt(bs / nsub);
    f[13] = (nsub * sxy - sx * sy) / (nsub * sxx - sx * sx);
    double ct = 0, ca = 0;
    for (int j = 0; j < k; ++j) {
        const double a2 = cf[2 * j] * cf[2 * j] + cf[2 * j + 1] * cf[2 * j + 1];
        ca += a2;
        if (j >= 24) ct += a2;
    }
    f[14] = 0.5 * std::log10(std::max(ct, 1e-300) / ca);
    f[15] = ist.rhi_iters[0];
    for (int i = 0; i < NK_MLP_IN; ++i) {
        if (!std::isfinite(f[i])) return fail(c, NK_EINVAL, "non-finite predictor feature");
        features[i] = (float)f[i];
    }
    return NK_OK;
}

int nk_predict_sizes(nk_ctx* c, nk_mlp* m, const double* b_dev, int k_max, int* k, int* ell, void* stream) {
    if (!c || !m || !b_dev || !k || !ell) return c ? fail(c, NK_EINVAL, "null pointer") : NK_EINVAL;
    if (k_max < 64 || k_max > nk::kMaxInnerK || (k_max & 1)) return fail(c, NK_EINVAL, "bad k_max");
    float f[NK_MLP_IN], y[NK_MLP_OUT];
    int rc = nk_features(c, b_dev, f, stream);
    if (rc) return rc;
    rc = nk_mlp_forward(m, f, 1, y);
    if (rc) return fail(c, rc, std::string("predictor: ") + nk_mlp_last_error(m));
    auto even = [](double v) { return 2 * (int)std::lround(0.5 * v); };
    const double kp = std::exp2(std::min(std::max((double)y[0], 0.0), 12.0));
    const double lp = std::exp2(std::min(std::max((double)y[1], 0.0), 12.0));
    int kk = std::min(std::max(even(kp), 64), k_max);
    int ll = std::min(std::max(even(lp), 16), std::min(kk, 256));
    *k = kk;
    *ell = ll;
    return NK_OK;
}

int nk_set_predictor(nk_ctx* c, nk_mlp* m) {
    if (!c) return NK_EINVAL;
    c->predictor = m;
    return NK_OK;
}

int nk_wait(nk_ctx* c, nk_stats* stats) {
    if (!c) return NK_EINVAL;
    if (!c->pending.on) return NK_OK;
    nk_ctx::Pending P = c->pending;
    c->pending.on = false;
    NK_CUDA(c, cudaSetDevice(c->device));
    const int n = P.n_rhs;
    std::vector<int> status(n), iters(n), kused(n, P.k), notconv(n, 0);
    std::vector<double> pv(n), zmin(n), zmax(n), xn(n);
    NK_CUDA(c, cudaMemcpyAsync(status.data(), P.status, sizeof(int) * n, cudaMemcpyDeviceToHost, P.st));
    NK_CUDA(c, cudaMemcpyAsync(iters.data(), P.iters, sizeof(int) * n, cudaMemcpyDeviceToHost, P.st));
    NK_CUDA(c, cudaMemcpyAsync(pv.data(), P.p, sizeof(double) * n, cudaMemcpyDeviceToHost, P.st));
    NK_CUDA(c, cudaMemcpyAsync(zmin.data(), P.zmin, sizeof(double) * n, cudaMemcpyDeviceToHost, P.st));
    NK_CUDA(c, cudaMemcpyAsync(zmax.data(), P.zmax, sizeof(double) * n, cudaMemcpyDeviceToHost, P.st));
    NK_CUDA(c, cudaMemcpyAsync(xn.data(), P.xnorm, sizeof(double) * n, cudaMemcpyDeviceToHost, P.st));
    NK_CUDA(c, cudaStreamSynchronize(P.st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, P.e0, P.e1);
    double tph[3];
    phase_times(c, P.e0, P.e1, tph);
    cudaEventDestroy(P.e0);
    cudaEventDestroy(P.e1);
    const int rc = collect_outcome(c, n, P.k, kused, notconv, 0, P.ell, P.launches, ms, status, iters, pv, zmin,
                                   zmax, xn, stats);
    if (stats) {
        stats->t_basis_ms = tph[0];
        stats->t_inner_ms = tph[1];
        stats->t_lift_ms = tph[2];
    }
    return rc;
}

const char* nk_last_error(const nk_ctx* c) { return c ? c->err.c_str() : "null context"; }

void nk_destroy(nk_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->pending.on) {
        cudaStreamSynchronize(c->pending.st);
        cudaEventDestroy(c->pending.e0);
        cudaEventDestroy(c->pending.e1);
    }
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.second.first);
    if (c->ws.p) cudaFree(c->ws.p);
    if (c->staging.p) cudaFree(c->staging.p);
    if (c->links_tmp.p) cudaFree(c->links_tmp.p);
    if (c->inner_tmp.p) cudaFree(c->inner_tmp.p);
    if (c->eps_buf.p) cudaFree(c->eps_buf.p);
    if (c->defl_buf.p) cudaFree(c->defl_buf.p);
    if (c->cg_buf.p) cudaFree(c->cg_buf.p);
    if (c->defl_L && c->defl_L != c->defl_R) cudaFree(c->defl_L);
    if (c->defl_R) cudaFree(c->defl_R);
    if (c->defl_neg) cudaFree(c->defl_neg);
    if (c->defl_sgn) cudaFree(c->defl_sgn);
    for (auto& e : c->ph)
        if (e) cudaEventDestroy(e);
    if (c->U64) cudaFree(c->U64);
    if (c->U32) cudaFree(c->U32);
    if (c->Udf) cudaFree(c->Udf);
    delete c;
}

}  // extern "C"
