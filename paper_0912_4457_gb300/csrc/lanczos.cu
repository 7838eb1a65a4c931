// Outer Krylov recurrence on the 12V-dimensional vectors, batched over RHS:
// Lanczos (App. A, mu = 0) and two-sided Lanczos (App. B, mu != 0), and the
// lift y = |x| V_k c (Eq. nested, App. C step 6).
//
// GB300 layout of the recurrence.  The basis is kept UNNORMALISED: the stored
// right vector is q_j = n_j v_j with n_0 = |x|, n_{j+1} = beta_j (so q_{j+1} is
// the residual r of step j itself), and the left vector p_j = m_j w_j with
// m_0 = |x|, m_{j+1} = gamma_j^*.  Every normalisation of App. A / B becomes a
// scalar folded into a coefficient, which removes the "v <- r / beta" pass
// and a third of the FP64 operations per vector element (FP64 is the scarce
// unit on GB300).  In exact arithmetic this is the paper's recurrence; the
// coefficients alpha, beta, gamma are the entries of H_k as App. A / B define
// them.  One outer step j is two kernels:
//   dslash_step1 (dslash.cu): s = A q_j / n_j (and t = A^dag p_j / m_j), then
//          r = s - (c_{j-1}/n_{j-1}) q_{j-1},  l = t - (beta^*_{j-1}/m_{j-1}) p_{j-1}
//          H(j,j) = v_j^dag r (= w_j^dag r two-sided), stored r -> q_{j+1}, l -> p_{j+1};
//   step2: r <- r - (H(j,j)/n_j) q_j,  l <- l - (H(j,j)^*/m_j) p_j,
//          beta = |r| (two-sided: delta = r^dag l, beta = sqrt(delta),
//          gamma = delta^*/beta; delta = 0 is a serious breakdown),
//          plus the FP32 copies the next mixed-precision stencil reads.
// In the mixed schedule, from the step where its recurrence turns two-float,
// both kernels work in two-float arithmetic on rings of the newest three
// right and left vectors (k_step2_df), and the basis columns they produce are
// stored as two-float values.
//
// Reductions are deterministic: a fixed grid, a fixed per-thread order,
// warp-shuffle and shared-memory block sums, per-block partials and a final
// fixed-order sum in the last block to finish (integer ticket, no
// floating-point atomics).  The same launch configuration therefore
// regenerates bit-identical coefficients, which the double-pass mode relies on.
#include "nk_common.cuh"
#include "nk_kernels.h"
#include "nk_tma.cuh"

namespace nk {

namespace {

constexpr int kThreads = 256;


__global__ void __launch_bounds__(kThreads) k_norm(Outer o, int keep_status) {
    __shared__ double2 sh[33];
    const int rhs = blockIdx.y;
    const double2* x = outer_q(o, rhs, 0);
    double acc = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < o.N; i += (long)o.nblk * blockDim.x) {
        double2 v = x[i];
        acc += v.x * v.x + v.y * v.y;
    }
    double2 part = block_sum(mk(acc, 0.0), sh);
    if (finish_partial(part, o.partials + (size_t)rhs * o.npart, o.counters + rhs, blockIdx.x, o.nblk)) {
        double2 tot = sum_partials(o.partials + (size_t)rhs * o.npart, o.nblk, sh);
        if (threadIdx.x == 0) {
            double nrm = sqrt(tot.x);
            o.xnorm[rhs] = nrm;
            // the second pass of NK_DOUBLE_PASS keeps a failure of the first
            // (breakdown, RHi): that source is not recomputed
            const int prev = o.status[rhs];
            const bool keep = keep_status && prev != kStatusOK && prev != kStatusZeroSource;
            o.status[rhs] = keep ? prev : (nrm > 0.0 ? kStatusOK : kStatusZeroSource);
            o.counters[rhs] = 0u;
            // scalars of step 0: n_0 = m_0 = |x|, no previous vector
            double2* sc = o.sc + (size_t)rhs * kScalars;
            const double2 inv = nrm > 0.0 ? cinv(mk(nrm, 0.0)) : mk(0.0, 0.0);
            sc[kScN] = inv;
            sc[kScC1] = mk(0.0, 0.0);
            sc[kScD] = inv;
            sc[kScM] = inv;
            sc[kScC1L] = mk(0.0, 0.0);
        }
    }
}

__device__ __forceinline__ dfc dfc_of(double2 v) {
    dfc r;
    r.x = df_from_double(v.x);
    r.y = df_from_double(v.y);
    return r;
}
__device__ __forceinline__ double2 double2_of(dfc v) { return mk(df_to_double(v.x), df_to_double(v.y)); }

// The next stencil's input copy of one element (FP32 or two-float), made on
// the integer pipe.  With the mixed schedule's rings the two-float copy is not
// made here (the FP64 steps write the rings themselves, which the two-float
// stencil reads).
// Element i = c V + s of RHS rhs (FP64 layout [12][V]); the FP32 copy goes to
// the pair layout.
__device__ __forceinline__ void put_copy(const Outer& o, int mode, bool left, int rhs, long i, double2 v) {
    if (mode == kCopy32) {
        const int V = (int)(o.N / 12);
        const int c = (int)(i / V), s = (int)(i - (long)c * V);
        float2 f = make_float2(d2f_int(v.x), d2f_int(v.y));
        reinterpret_cast<float2*>(left ? o.p32 : o.q32)[(size_t)rhs * o.N + f32_pair_index(c, s, V)] = f;
    } else if (mode == kCopyDF && !o.qr) {
        dfc w;
        w.x = df_from_double(v.x);
        w.y = df_from_double(v.y);
        (left ? o.pdf : o.qdf)[(size_t)rhs * o.N + i] = w;
    }
}

// q_0 = x is already in place; p_0 = x, and the copies the first stencil reads.
// Mixed schedule: the two-float rings hold q_0 and p_0, and a two-float
// stencil reads the ring itself.
__global__ void __launch_bounds__(kThreads) k_init(Outer o, int copy_mode) {
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const double2* x = outer_q(o, rhs, 0);
    double2* p = o.two_sided ? outer_p(o, rhs, 0) : nullptr;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < o.N; i += (long)o.nblk * blockDim.x) {
        double2 a = x[i];
        if (p) p[i] = a;
        put_copy(o, copy_mode, false, rhs, i, a);
        if (p) put_copy(o, copy_mode, true, rhs, i, a);
        if (o.qr) {
            const dfc d = dfc_of(a);
            ring_q(o, rhs, 0)[i] = d;
            if (o.two_sided) ring_p(o, rhs, 0)[i] = d;
        }
    }
}

// End of step 2: the deterministic reduction of the per-thread partial
// (r^dag r, or r^dag l two-sided) and, in the last block, beta and gamma and
// the scalars of step j + 1 (one complex division per warp, side by side on
// the SM sub-partitions).
template <bool TS>
__device__ __forceinline__ void step2_finish(const Outer& o, int rhs, int j, double2 acc, double2* sh) {
    __shared__ double2 bg[2];
    double2 part = block_sum(acc, sh);
    if (finish_partial(part, o.partials + (size_t)rhs * o.npart, o.counters + rhs, blockIdx.x, o.nblk)) {
        double2 d = sum_partials(o.partials + (size_t)rhs * o.npart, o.nblk, sh);
        if (threadIdx.x == 0) {
            const size_t at = (size_t)rhs * o.k + j;
            double2 b, g;
            if (!TS) {
                const double bb = sqrt(d.x);             // beta <- sqrt(r^dag r)
                b = g = mk(bb, 0.0);
                if (!(bb > 0.0) || !isfinite(bb)) mark_failed(o, rhs, kStatusBreakdown);
            } else if ((d.x == 0.0 && d.y == 0.0) || !isfinite(d.x) || !isfinite(d.y)) {
                // serious breakdown: delta = 0 (App. B); a non-finite delta is treated alike
                mark_failed(o, rhs, kStatusBreakdown);
                b = g = mk(0.0, 0.0);
            } else {
                b = csqrt_principal(d);                  // beta <- sqrt(delta)
                g = cdiv(cconj(d), b);                   // gamma <- delta^* / beta
            }
            o.beta[at] = b;
            o.gamma[at] = g;
            bg[0] = b;
            bg[1] = g;
            o.counters[rhs] = 0u;
        }
        __syncthreads();
        // step j + 1: n_{j+1} = beta_j, m_{j+1} = gamma_j^*
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0 && w < 5 && j + 1 < o.k && o.status[rhs] == kStatusOK) {
            const double2 b = bg[0], g = bg[1];
            double2* sc = o.sc + (size_t)rhs * kScalars;
            if (w == 0) sc[kScN] = cinv(b);
            else if (w == 1) sc[kScC1] = cdiv(TS ? g : b, scale_n(o, rhs, j));
            else if (w == 2) sc[kScD] = TS ? cinv(g) : cinv(b);
            else if (w == 3) sc[kScM] = cinv(cconj(g));
            else sc[kScC1L] = cdiv(cconj(b), scale_m(o, rhs, j));
        }
    }
}

// ---- streaming FP64 kernels of the FP64 recurrence ----------------------------
// Step 1 (after the FP32 stencil) and step 2 stream their operand vectors
// through shared memory with bulk asynchronous copies (the TMA engine,
// cp.async.bulk, nk_tma.cuh).  A CTA owns a contiguous range of sites of one
// RHS and walks it in tiles of kTile sites.  Warp w owns component pair w
// (spin-colour components 2w and 2w + 1: rows 2w, 2w + 1 of an FP64 vector,
// row w of an FP32 pair-layout vector) and runs its own pipeline: kStages
// stage buffers with their own mbarriers, into which its lanes copy the
// warp's rows of every operand vector for a tile, kStages - 1 tiles ahead of
// its arithmetic; lane l then takes site s0 + l of the tile and writes its
// results straight to global memory.  No CTA-wide barrier inside the loop:
// the warps run independently.  GB300's FP64 pipe (about 0.6 T DFMA/s) is
// kept busy by a few warps per SM as long as they have operands; the copies
// keep enough bytes in flight for HBM without holding them in registers.
constexpr int kTile = 32;                       // sites per tile = lanes of a warp
constexpr int kStreamWarps = 6;                 // one per component pair
constexpr int kStreamThreads = 32 * kStreamWarps;
constexpr int kStages = 2;
constexpr int kRowBytes = kTile * 16;           // one row of a tile: kTile 16-byte elements
constexpr int kStep2Rows = 8;                   // rows of one warp's stage: step 2
constexpr int kStep1Rows = 8;                   // step 1 after the FP32 stencil
constexpr int kStep1Rows64 = 10;                // step 1 after the two-float stencil (FP64 s, t)

// One operand vector of a streaming kernel (row r of V 16-byte elements at
// base + r V 16 bytes): rows = 2 for an FP64 vector (warp w reads rows 2w,
// 2w + 1), 1 for an FP32 pair-layout vector (row w), 0 for an absent operand.
struct TileStream {
    const char* base;
    int rows;
};

// The copies of warp w for the tile of sites [s0, s0 + n): one row per lane
// (the rows of stream k follow those of streams 0 .. k-1 in the stage),
// armed on bar with their byte count by lane 0.
template <int NS>
__device__ __forceinline__ void issue_warp_tile(const TileStream (&ts)[NS], char* stage, uint64_t* bar, unsigned V,
                                                unsigned s0, unsigned n, int w, int lane) {
    int total = 0;
#pragma unroll
    for (int k = 0; k < NS; ++k) total += ts[k].rows;
    const unsigned bytes = n * 16u;
    if (lane == 0) {
        fence_proxy_async_smem();   // the stage was last read through the generic proxy
        mbar_arrive_expect_tx(bar, (unsigned)total * bytes);
    }
    __syncwarp();
    int off = 0;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const int rows = ts[k].rows;
        if (lane >= off && lane < off + rows) {
            const unsigned row = (unsigned)(w * rows + lane - off);
            bulk_copy_g2s(stage + (size_t)lane * kRowBytes, ts[k].base + ((size_t)row * V + s0) * 16, bytes, bar);
        }
        off += rows;
    }
}

// The tile loop of warp w over the site range of CTA blockIdx.x (of o.nblk per
// RHS): f(stage, s0, n) on each tile once its copies have landed.  Returns
// false if a wait ran out (the warp's copies still in flight are then waited
// for, bounded, before returning).
template <int ROWS, int NS, typename F>
__device__ __forceinline__ bool stream_tiles(const Outer& o, const TileStream (&ts)[NS], F&& f) {
    extern __shared__ __align__(128) char smem[];
    __shared__ uint64_t bar[kStreamWarps][kStages];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned V = (unsigned)(o.N / 12);
    const unsigned s_lo = (unsigned)((unsigned long long)blockIdx.x * V / (unsigned)o.nblk);
    const unsigned s_hi = (unsigned)((unsigned long long)(blockIdx.x + 1) * V / (unsigned)o.nblk);
    const int ntiles = (int)((s_hi - s_lo + kTile - 1) / kTile);
    const size_t stage_bytes = (size_t)ROWS * kRowBytes;   // ROWS >= the streams' rows
    char* mine = smem + (size_t)w * kStages * stage_bytes;
    uint64_t* mbar = bar[w];
    if (lane == 0) {
#pragma unroll
        for (int st = 0; st < kStages; ++st) mbar_init(&mbar[st], 1);
        mbar_init_fence();
    }
    __syncwarp();
    for (int t = 0; t < kStages - 1 && t < ntiles; ++t) {
        const unsigned s0 = s_lo + t * kTile;
        issue_warp_tile(ts, mine + t * stage_bytes, &mbar[t], V, s0, min((unsigned)kTile, s_hi - s0), w, lane);
    }
    int t = 0;
    bool ok = true;
    for (; t < ntiles; ++t) {
        // the tile kStages - 1 ahead goes into the stage freed by tile t - 1
        const int ahead = t + kStages - 1;
        if (ahead < ntiles) {
            const unsigned s0 = s_lo + ahead * kTile;
            issue_warp_tile(ts, mine + (ahead % kStages) * stage_bytes, &mbar[ahead % kStages], V, s0,
                            min((unsigned)kTile, s_hi - s0), w, lane);
        }
        const int st = t % kStages;
        ok = __all_sync(0xffffffffu, mbar_wait_bounded(&mbar[st], (unsigned)(t / kStages) & 1u, kWaitLimitNs));
        if (!ok) break;
        const unsigned s0 = s_lo + t * kTile;
        f(mine + st * stage_bytes, s0, min((unsigned)kTile, s_hi - s0));
        __syncwarp();   // every lane is done with the stage before it is refilled
    }
    if (ok) return true;
    if (lane == 0)   // copies issued for tiles t .. t + kStages - 1
        for (int u = t; u < ntiles && u < t + kStages; ++u)
            mbar_wait_bounded(&mbar[u % kStages], (unsigned)(u / kStages) & 1u, kWaitLimitNs);
    __syncwarp();
    return false;
}

// The FP64 loops take no negated operand: in a throughput test on GB300 a
// DFMA with a negated multiplicand ran at 85% of the rate of a plain one.  The
// negated scalars are formed once per kernel by flipping the sign bit, and
// the imaginary part of an inner product sums its two products separately.
__device__ __forceinline__ double neg_bits(double x) {
    return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}
__device__ __forceinline__ double2 neg_bits(double2 c) { return mk(neg_bits(c.x), neg_bits(c.y)); }
// s - c p, with nc = -c
__device__ __forceinline__ double2 cfma_sub(double2 s, double2 c, double2 nc, double2 p) {
    return mk(fma(nc.x, p.x, fma(c.y, p.y, s.x)), fma(nc.x, p.y, fma(nc.y, p.x, s.y)));
}
// s + c p, with nc = -c
__device__ __forceinline__ double2 cfma_add(double2 s, double2 c, double2 nc, double2 p) {
    return mk(fma(c.x, p.x, fma(nc.y, p.y, s.x)), fma(c.x, p.y, fma(c.y, p.x, s.y)));
}
// conj(a) b accumulated as (re, im+, im-): im = im+ - im-
struct Dot3 {
    double re, ip, im;
};
__device__ __forceinline__ void dot3_add(Dot3& d, double2 a, double2 b) {
    d.re = fma(a.x, b.x, fma(a.y, b.y, d.re));
    d.ip = fma(a.x, b.y, d.ip);
    d.im = fma(a.y, b.x, d.im);
}

// FP64 step 2 (the recurrence of NK_FP64 and of the mixed schedule):
//   r <- r - (H(j,j)/n_j) q_j,  l <- l - (H(j,j)^*/m_j) p_j,  delta += r^dag l,
// plus the copies the next stencil reads (FP32 pair layout; write_ring: also
// two-float copies in the rings for a two-float stencil or a later ring
// step).  Stage rows of warp w (components 2w + h): q_j h, r 2 + h, p_j 4 + h,
// l 6 + h.
template <bool TS>
__global__ void __launch_bounds__(kStreamThreads) k_step2(Outer o, int j, int copy_mode, int write_ring) {
    __shared__ double2 sh[33];
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const double2 c3 = o.sc[(size_t)rhs * kScalars + kScC3];
    const double2 c4 = o.sc[(size_t)rhs * kScalars + kScC4];
    const unsigned V = (unsigned)(o.N / 12);
    const double2* qj = outer_q(o, rhs, j);
    double2* r = outer_q(o, rhs, j + 1);
    const double2* pj = TS ? outer_p(o, rhs, j) : nullptr;
    double2* l = TS ? outer_p(o, rhs, j + 1) : nullptr;
    float4* __restrict__ r32 = o.q32 + (size_t)rhs * 6 * V;
    float4* __restrict__ l32 = TS ? o.p32 + (size_t)rhs * 6 * V : nullptr;
    dfc* __restrict__ rr_ring = write_ring ? ring_q(o, rhs, j + 1) : nullptr;
    dfc* __restrict__ ll_ring = (write_ring && TS) ? ring_p(o, rhs, j + 1) : nullptr;
    const TileStream ts[4] = {{(const char*)qj, 2}, {(const char*)r, 2}, {(const char*)pj, TS ? 2 : 0},
                              {(const char*)l, TS ? 2 : 0}};
    const double2 nc3 = neg_bits(c3), nc4 = neg_bits(c4);
    const int cp = threadIdx.x >> 5, sl = threadIdx.x & 31;
    Dot3 acc = {0.0, 0.0, 0.0};
    const bool ok = stream_tiles<kStep2Rows>(o, ts, [&](const char* stage, unsigned s0, unsigned n) {
        if ((unsigned)sl >= n) return;
        const double2* sv = reinterpret_cast<const double2*>(stage);
        double2 rv[2], lv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = 2 * cp + h;
            const size_t e = (size_t)c * V + s0 + sl;
            const double2 q = sv[h * kTile + sl], a0 = sv[(2 + h) * kTile + sl];
            // r <- r - c3 q, l <- l - c4 p with explicit FMA
            const double2 a = TS ? cfma_sub(a0, c3, nc3, q) : mk(fma(nc3.x, q.x, a0.x), fma(nc3.x, q.y, a0.y));
            rv[h] = a;
            r[e] = a;
            if (rr_ring) rr_ring[e] = dfc_of(a);
            if (TS) {
                const double2 b = cfma_sub(sv[(6 + h) * kTile + sl], c4, nc4, sv[(4 + h) * kTile + sl]);
                lv[h] = b;
                l[e] = b;
                if (ll_ring) ll_ring[e] = dfc_of(b);
                dot3_add(acc, a, b);   // conj(r) l
            } else {
                acc.re = fma(a.x, a.x, fma(a.y, a.y, acc.re));
            }
        }
        if (copy_mode == kCopy32) {
            const size_t f = (size_t)cp * V + s0 + sl;
            r32[f] = make_float4(d2f_int(rv[0].x), d2f_int(rv[0].y), d2f_int(rv[1].x), d2f_int(rv[1].y));
            if (TS) l32[f] = make_float4(d2f_int(lv[0].x), d2f_int(lv[0].y), d2f_int(lv[1].x), d2f_int(lv[1].y));
        }
    });
    double2 tot = mk(acc.re, acc.ip - acc.im);
    if (!ok) {
        if (threadIdx.x == 0) mark_failed(o, rhs, kStatusTimeout);
        tot = mk(0.0, 0.0);
    }
    step2_finish<TS>(o, rhs, j, tot, sh);
}

// FP64 step 1 of the FP32- and two-float-stencil steps of an FP64
// recurrence, after the multi-RHS stencil has left s = (A q_j)/n_j and
// t = (A^dag p_j)/m_j in o.s32 (FP32, pair layout) or, S64, in o.s64 (FP64
// from the two-float stencil):
//   r = s - (c_{j-1}/n_{j-1}) q_{j-1} -> q_{j+1},
//   l = t - (beta^*_{j-1}/m_{j-1}) p_{j-1} -> p_{j+1}   (two-sided, not at the last step),
//   H(j,j) = (p_j^dag r) / m_j^*  (Hermitian: Re(q_j^dag r) / n_j),
// an FP32 stencil output entering the FP64 arithmetic exactly (FP32 -> FP64
// on the integer pipe).  The finishing block forms H(j,j) and the step-2
// scalars.  PASS2 (the second pass of NK_DOUBLE_PASS) also accumulates
// y += c'_j q_j.  Stage rows of warp w (components 2w + h), with
// F = 1 (FP32 s: one row of pairs) or 2 (FP64 s: rows h): s 0 .. F - 1,
// q_{j-1} F + h, dot vector (p_j, or q_j Hermitian) F + 2 + h, then two-sided
// and not at the last step t F + 4 .., p_{j-1} 2 F + 4 + h.
template <bool TS, bool PASS2, bool S64>
__global__ void __launch_bounds__(kStreamThreads) k_step1(Outer o, int j) {
    __shared__ double2 sh[33];
    constexpr int F = S64 ? 2 : 1;
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const double2* sc = o.sc + (size_t)rhs * kScalars;
    const double2 c1 = sc[kScC1], c1l = sc[kScC1L];
    const unsigned V = (unsigned)(o.N / 12);
    const int jp = j > 0 ? j - 1 : j;   // c1 = 0 at j = 0
    const bool left = TS && j < o.k - 1;   // the last step makes no new left vector
    const char* s_in = S64 ? (const char*)(o.s64 + (size_t)rhs * o.N) : (const char*)(o.s32 + (size_t)rhs * 6 * V);
    const char* t_in = S64 ? (const char*)(o.s64 + (size_t)(o.n_rhs + rhs) * o.N)
                           : (const char*)(o.s32 + (size_t)(o.n_rhs + rhs) * 6 * V);
    const double2* qprev = outer_q(o, rhs, jp);
    const double2* pprev = TS ? outer_p(o, rhs, jp) : nullptr;
    const double2* dotv = TS ? outer_p(o, rhs, j) : outer_q(o, rhs, j);
    double2* __restrict__ rn = outer_q(o, rhs, j + 1);
    double2* __restrict__ ln = left ? outer_p(o, rhs, j + 1) : nullptr;
    double2* __restrict__ yacc = PASS2 ? o.y + (size_t)rhs * o.N : nullptr;
    const double2 cpj = PASS2 ? o.cp[(size_t)rhs * o.k + j] : mk(0.0, 0.0);
    const double2* __restrict__ qj = outer_q(o, rhs, j);
    const TileStream ts[5] = {{s_in, F}, {(const char*)qprev, 2}, {(const char*)dotv, 2},
                              {t_in, left ? F : 0}, {(const char*)pprev, left ? 2 : 0}};
    const double2 nc1 = neg_bits(c1), nc1l = neg_bits(c1l), ncpj = neg_bits(cpj);
    const int cp = threadIdx.x >> 5, sl = threadIdx.x & 31;
    Dot3 acc = {0.0, 0.0, 0.0};
    const bool ok = stream_tiles<S64 ? kStep1Rows64 : kStep1Rows>(o, ts, [&](const char* stage, unsigned s0,
                                                                                unsigned n) {
        if ((unsigned)sl >= n) return;
        const double2* sv = reinterpret_cast<const double2*>(stage);
        const float4* sf = reinterpret_cast<const float4*>(stage);
        float4 sv4 = make_float4(0.f, 0.f, 0.f, 0.f), tv4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!S64) {
            sv4 = sf[sl];
            if (left) tv4 = sf[(F + 4) * kTile + sl];
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = 2 * cp + h;
            const size_t e = (size_t)c * V + s0 + sl;
            double2 rr;
            if (S64) {
                rr = sv[h * kTile + sl];
            } else {
                const float2 s2 = h ? make_float2(sv4.z, sv4.w) : make_float2(sv4.x, sv4.y);
                rr = mk(f2d_int(s2.x), f2d_int(s2.y));
            }
            const double2 qv = sv[(F + h) * kTile + sl];
            rr = TS ? cfma_sub(rr, c1, nc1, qv) : mk(fma(nc1.x, qv.x, rr.x), fma(nc1.x, qv.y, rr.y));
            rn[e] = rr;
            const double2 d = sv[(F + 2 + h) * kTile + sl];
            if (TS) dot3_add(acc, d, rr);   // conj(d) r
            else acc.re = fma(d.x, rr.x, fma(d.y, rr.y, acc.re));
            if (left) {
                double2 tt;
                if (S64) {
                    tt = sv[(F + 4 + h) * kTile + sl];
                } else {
                    const float2 t2 = h ? make_float2(tv4.z, tv4.w) : make_float2(tv4.x, tv4.y);
                    tt = mk(f2d_int(t2.x), f2d_int(t2.y));
                }
                ln[e] = cfma_sub(tt, c1l, nc1l, sv[(2 * F + 4 + h) * kTile + sl]);
            }
            if (PASS2) yacc[e] = cfma_add(yacc[e], cpj, ncpj, qj[e]);
        }
    });
    double2 tot = mk(acc.re, acc.ip - acc.im);
    if (!ok) {
        if (threadIdx.x == 0) mark_failed(o, rhs, kStatusTimeout);
        tot = mk(0.0, 0.0);
    }
    const double2 part = block_sum(tot, sh);
    if (finish_partial(part, o.partials + (size_t)rhs * o.npart, o.counters + rhs, blockIdx.x, o.nblk)) {
        const double2 a = sum_partials(o.partials + (size_t)rhs * o.npart, o.nblk, sh);
        // Hermitian: H(j,j) = Re(q_j^dag r) / n_j, real (App. C); two-sided: (p_j^dag r) / m_j^*
        const double2 al = TS ? cmul(sc[kScD], a) : mk(a.x * sc[kScD].x, 0.0);
        const int w = threadIdx.x >> 5;
        if (threadIdx.x == 0) {
            o.alpha[(size_t)rhs * o.k + j] = al;
            o.counters[rhs] = 0u;
        }
        // the step-2 scalars H(j,j)/n_j and H(j,j)^*/m_j, one division per warp
        if ((threadIdx.x & 31) == 0 && w == 1) o.sc[(size_t)rhs * kScalars + kScC3] = cdiv(al, scale_n(o, rhs, j));
        if ((threadIdx.x & 31) == 0 && w == 2)
            o.sc[(size_t)rhs * kScalars + kScC4] = TS ? cdiv(cconj(al), scale_m(o, rhs, j)) : mk(0.0, 0.0);
    }
}

size_t step2_smem() { return (size_t)kStreamWarps * kStages * kStep2Rows * kRowBytes; }
size_t step1_smem(bool s64) { return (size_t)kStreamWarps * kStages * (s64 ? kStep1Rows64 : kStep1Rows) * kRowBytes; }

// Step 2 of the late (FP32-stencil) steps of the mixed schedule in two-float
// arithmetic on the FP32 pipe, on the two-float rings: r and l (left in ring slot j + 1
// by the stencil kernel) are updated with q_j and p_j from the rings; r is
// also written to the basis Q (as two-float values in a single-pass solve,
// else FP64: one FP64 addition per component), and the
// FP32 copy the next FP32 stencil reads is the high part (a two-float
// stencil reads the ring).  The FP32 stencil of the late steps perturbs the
// recurrence at 1e-7; 48-bit arithmetic adds about 1e-14.  The all-FP64
// schedule (NK_FP64) keeps k_step2.
template <bool TS>
__global__ void __launch_bounds__(kThreads, 2) k_step2_df(Outer o, int j, int copy_mode) {
    __shared__ double2 sh[33];
    const int rhs = blockIdx.y;
    if (o.status[rhs] != kStatusOK) return;
    const dfc c3 = dfc_of(o.sc[(size_t)rhs * kScalars + kScC3]);
    const dfc c4 = dfc_of(o.sc[(size_t)rhs * kScalars + kScC4]);
    const int V = (int)(o.N / 12);
    const dfc* __restrict__ qj = ring_q(o, rhs, j);
    dfc* __restrict__ r = ring_q(o, rhs, j + 1);
    double2* __restrict__ rq = outer_q(o, rhs, j + 1);
    const bool qdf = j + 1 >= o.q_df_from;   // the basis column is kept in two-float form
    const dfc* __restrict__ pj = TS ? ring_p(o, rhs, j) : nullptr;
    dfc* __restrict__ l = TS ? ring_p(o, rhs, j + 1) : nullptr;
    const size_t vb = (size_t)rhs * o.N;
    // U elements per thread and iteration, all their loads issued before any
    // arithmetic (the kernel is bound by the latency of these L2 reads), one
    // accumulator each
    constexpr int U = 4;
    df ax[U], ay[U];
#pragma unroll
    for (int u = 0; u < U; ++u) ax[u] = ay[u] = df(0);
    const long stride = (long)o.nblk * blockDim.x;
    for (long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x; i0 < o.N; i0 += U * stride) {
        dfc q[U], rr[U], pv[U], ll[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long i = i0 + u * stride;
            if (i < o.N) {
                q[u] = qj[i];
                rr[u] = r[i];
                if (TS) { pv[u] = pj[i]; ll[u] = l[i]; }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long i = i0 + u * stride;
            if (i >= o.N) break;
            // r <- r - c3 q, l <- l - c4 p
            dfc& a = rr[u];
            if (TS) {
                a.x = a.x - (c3.x * q[u].x - c3.y * q[u].y);
                a.y = a.y - (c3.x * q[u].y + c3.y * q[u].x);
            } else {
                a.x = a.x - c3.x * q[u].x;
                a.y = a.y - c3.x * q[u].y;
            }
            r[i] = a;
            if (qdf) reinterpret_cast<dfc*>(rq)[i] = a;
            else rq[i] = double2_of(a);
            const int c = (int)(i / V), site = (int)(i - (long)c * V);
            const size_t i32 = vb + f32_pair_index(c, site, V);
            if (copy_mode == kCopy32) reinterpret_cast<float2*>(o.q32)[i32] = make_float2(a.x.hi, a.y.hi);
            if (TS) {
                dfc& b = ll[u];
                b.x = b.x - (c4.x * pv[u].x - c4.y * pv[u].y);
                b.y = b.y - (c4.x * pv[u].y + c4.y * pv[u].x);
                l[i] = b;
                if (copy_mode == kCopy32) reinterpret_cast<float2*>(o.p32)[i32] = make_float2(b.x.hi, b.y.hi);
                ax[u] += a.x * b.x + a.y * b.y;   // conj(r) l
                ay[u] += a.x * b.y - a.y * b.x;
            } else {
                ax[u] += a.x * a.x + a.y * a.y;
            }
        }
    }
    step2_finish<TS>(o, rhs, j, mk(df_to_double((ax[0] + ax[1]) + (ax[2] + ax[3])),
                                   df_to_double((ay[0] + ay[1]) + (ay[2] + ay[3]))), sh);
}

// c'_j = |x| c_j / n_j: the lift coefficients on the unnormalised basis
// (zero from kused on, where the basis and its scales were never computed).
__global__ void k_lift_coef(Outer o, const double2* __restrict__ c, const int* __restrict__ kused,
                            double2* __restrict__ cp) {
    const int rhs = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= o.k) return;
    double2* out = cp + (size_t)rhs * o.k;
    if (o.status[rhs] != kStatusOK || j >= kused[rhs]) { out[j] = mk(0.0, 0.0); return; }
    out[j] = cscale(cdiv(c[(size_t)rhs * o.k + j], scale_n(o, rhs, j)), o.xnorm[rhs]);
}

// per RHS: dn = (|c - c_prev|, |c|) over the first k entries; then c_prev <- c
__global__ void k_adapt_delta(Outer o, const double2* __restrict__ c, double2* __restrict__ cprev, int k,
                              double2* __restrict__ dn) {
    __shared__ double2 sh[33];
    const int rhs = blockIdx.x;
    if (o.status[rhs] != kStatusOK) return;   // frozen or failed: keep its accepted c
    const double2* cr = c + (size_t)rhs * o.k;
    double2* pr = cprev + (size_t)rhs * o.k;
    double d = 0.0, n = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double2 a = cr[j], b = pr[j];
        d += cnorm2(csub(a, b));
        n += cnorm2(a);
    }
    double2 t = block_sum(mk(d, n), sh);
    for (int j = threadIdx.x; j < k; j += blockDim.x) pr[j] = cr[j];
    if (threadIdx.x == 0) dn[rhs] = mk(sqrt(t.x), sqrt(t.y));
}

// y_r = sum_j c'_r[j] q_j  (reads every basis vector once)
__global__ void __launch_bounds__(kThreads) k_lift(Outer o, const double2* __restrict__ cp,
                                                    const int* __restrict__ kused, double2* __restrict__ y) {
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= o.N) return;
    double2* yo = y + (size_t)rhs * o.N;
    if (o.status[rhs] != kStatusOK) { yo[i] = mk(0.0, 0.0); return; }
    const double2* cr = cp + (size_t)rhs * o.k;
    const double2* Qr = o.Q + (size_t)rhs * o.qcols * o.N;
    const int ku = kused[rhs];
    // two FMA per real part (`acc += a * b - c * d` would be a multiply, a fused
    // multiply-add and an add on the FP64 pipe)
    double2 acc = mk(0.0, 0.0);
#pragma unroll 4
    for (int j = 0; j < ku; ++j) {
        const double2 cj = __ldg(cr + j);
        const double2 v = Qr[(size_t)j * o.N + i];
        acc.x = fma(cj.x, v.x, fma(neg_bits(cj.y), v.y, acc.x));
        acc.y = fma(cj.x, v.y, fma(cj.y, v.x, acc.y));
    }
    yo[i] = acc;
}

// The same lift in two-float arithmetic for the mixed schedule: the
// coefficients are converted once per block into shared memory, each basis
// element on load, and the sum runs in two accumulators (even and odd j).
__global__ void __launch_bounds__(kThreads) k_lift_df(Outer o, const double2* __restrict__ cp,
                                                       const int* __restrict__ kused, double2* __restrict__ y) {
    extern __shared__ dfc cs[];   // [kused]
    const int rhs = blockIdx.y;
    const int ku = kused[rhs];
    const double2* cr = cp + (size_t)rhs * o.k;
    for (int j = threadIdx.x; j < ku; j += blockDim.x) cs[j] = dfc_of(cr[j]);
    __syncthreads();
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= o.N) return;
    double2* yo = y + (size_t)rhs * o.N;
    if (o.status[rhs] != kStatusOK) { yo[i] = mk(0.0, 0.0); return; }
    const double2* Qr = o.Q + (size_t)rhs * o.qcols * o.N;
    dfc acc[2];
    acc[0].x = df(0); acc[0].y = df(0); acc[1] = acc[0];
    const int j1 = min(ku, o.q_df_from);   // columns [j1, ku) are two-float already
    for (int j = 0; j < ku; ++j) {
        const dfc c = cs[j];
        const dfc v = j < j1 ? dfc_of(Qr[(size_t)j * o.N + i]) : reinterpret_cast<const dfc*>(Qr)[(size_t)j * o.N + i];
        dfc& a = acc[j & 1];
        a.x += c.x * v.x - c.y * v.y;
        a.y += c.x * v.y + c.y * v.x;
    }
    dfc t;
    t.x = acc[0].x + acc[1].x;
    t.y = acc[0].y + acc[1].y;
    yo[i] = double2_of(t);
}

// double pass: zero the status of sources that are exactly zero
__global__ void k_zero_bad(Outer o, double2* y) {
    const int rhs = blockIdx.y;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= o.N) return;
    if (o.status[rhs] != kStatusOK) y[(size_t)rhs * o.N + i] = mk(0.0, 0.0);
}

}  // namespace

void launch_outer_init(const Outer& o, int copy_mode, cudaStream_t st, bool keep_status) {
    dim3 grid(o.nblk, o.n_rhs);
    k_norm<<<grid, kThreads, 0, st>>>(o, keep_status ? 1 : 0);
    k_init<<<grid, kThreads, 0, st>>>(o, copy_mode);
}

void launch_outer_step1(const Outer& o, int j, bool s64, cudaStream_t st) {
    dim3 grid(o.nblk, o.n_rhs);
    const bool pass2 = o.y != nullptr;
    const size_t sm = step1_smem(s64);
#define NK_STEP1(TS_, P2_, S_) k_step1<TS_, P2_, S_><<<grid, kStreamThreads, sm, st>>>(o, j)
    if (o.two_sided) {
        if (pass2) { if (s64) NK_STEP1(true, true, true); else NK_STEP1(true, true, false); }
        else { if (s64) NK_STEP1(true, false, true); else NK_STEP1(true, false, false); }
    } else {
        if (pass2) { if (s64) NK_STEP1(false, true, true); else NK_STEP1(false, true, false); }
        else { if (s64) NK_STEP1(false, false, true); else NK_STEP1(false, false, false); }
    }
#undef NK_STEP1
}

// CTAs of the two-sided step-2 kernel that fit one SM (its stage buffers
// decide), queried once per device after lanczos_init_attributes.
int stream_ctas_per_sm() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2<true>, kStreamThreads, step2_smem()) !=
                cudaSuccess || n < 1) {
            cudaGetLastError();
            return 1;   // attributes not set yet: not cached
        }
        cached[dev] = n;
    }
    return cached[dev];
}

int stream_tile_sites() { return kTile; }

void lanczos_init_attributes() {
    // dynamic shared memory above 48 KB for the stage buffers of the streaming
    // kernels, and the largest shared-memory carveout so that several CTAs fit an SM
    const int carve = cudaSharedmemCarveoutMaxShared;
#define NK_ATTR(K_, SM_)                                                                    \
    cudaFuncSetAttribute(K_, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(SM_));     \
    cudaFuncSetAttribute(K_, cudaFuncAttributePreferredSharedMemoryCarveout, carve)
    NK_ATTR(k_step2<true>, step2_smem());
    NK_ATTR(k_step2<false>, step2_smem());
    NK_ATTR((k_step1<true, true, false>), step1_smem(false));
    NK_ATTR((k_step1<true, false, false>), step1_smem(false));
    NK_ATTR((k_step1<false, true, false>), step1_smem(false));
    NK_ATTR((k_step1<false, false, false>), step1_smem(false));
    NK_ATTR((k_step1<true, true, true>), step1_smem(true));
    NK_ATTR((k_step1<true, false, true>), step1_smem(true));
    NK_ATTR((k_step1<false, true, true>), step1_smem(true));
    NK_ATTR((k_step1<false, false, true>), step1_smem(true));
#undef NK_ATTR
}

void launch_outer_step2(const Outer& o, int j, int copy_mode, bool ring, bool write_ring, cudaStream_t st) {
    dim3 grid(o.nblk, o.n_rhs);
    const int wr = (write_ring && o.qr) ? 1 : 0;
    if (!ring || !o.qr) {   // FP64 step
        const size_t sm = step2_smem();
        if (o.two_sided) k_step2<true><<<grid, kStreamThreads, sm, st>>>(o, j, copy_mode, wr);
        else k_step2<false><<<grid, kStreamThreads, sm, st>>>(o, j, copy_mode, wr);
    } else {
        if (o.two_sided) k_step2_df<true><<<grid, kThreads, 0, st>>>(o, j, copy_mode);
        else k_step2_df<false><<<grid, kThreads, 0, st>>>(o, j, copy_mode);
    }
}

void launch_lift_coef(const Outer& o, const double2* c, const int* kused, double2* cp, cudaStream_t st) {
    dim3 grid((o.k + 127) / 128, o.n_rhs);
    k_lift_coef<<<grid, 128, 0, st>>>(o, c, kused, cp);
}

void launch_lift(const Outer& o, const double2* cp, const int* kused, double2* y, cudaStream_t st) {
    dim3 grid((unsigned)((o.N + kThreads - 1) / kThreads), o.n_rhs);
    // the two-float lift only where the two-float recurrence wrote two-float
    // basis columns; an FP64 recurrence is lifted in FP64
    if (o.q_ring) k_zero_bad<<<grid, kThreads, 0, st>>>(o, y);
    else if (o.qr && o.q_df_from < o.k) k_lift_df<<<grid, kThreads, sizeof(dfc) * (size_t)o.k, st>>>(o, cp, kused, y);
    else k_lift<<<grid, kThreads, 0, st>>>(o, cp, kused, y);
}

__global__ void k_fill_int(int* p, int n, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

void launch_fill_int(int* p, int n, int value, cudaStream_t st) {
    k_fill_int<<<(n + 127) / 128, 128, 0, st>>>(p, n, value);
}

// per RHS r: (|x2_r - b_r|^2, |b_r|^2), one block per RHS, fixed-order sums
__global__ void k_eps_sums(const double2* __restrict__ b, const double2* __restrict__ x2, long N,
                           double2* __restrict__ out) {
    __shared__ double2 sh[33];
    const size_t base = (size_t)blockIdx.x * N;
    double d = 0.0, n = 0.0;
    for (long i = threadIdx.x; i < N; i += blockDim.x) {
        const double2 a = b[base + i], c = x2[base + i];
        d += cnorm2(csub(c, a));
        n += cnorm2(a);
    }
    const double2 t = block_sum(mk(d, n), sh);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
}

void launch_eps_sums(const double2* b, const double2* x2, int n, long N, double2* out, cudaStream_t st) {
    k_eps_sums<<<n, 1024, 0, st>>>(b, x2, N, out);
}

void launch_adapt_delta(const Outer& o, const double2* c, double2* c_prev, int k, double2* dn, cudaStream_t st) {
    k_adapt_delta<<<o.n_rhs, 256, 0, st>>>(o, c, c_prev, k, dn);
}

}  // namespace nk
