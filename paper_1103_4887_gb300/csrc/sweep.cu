// The hot path: one persistent cooperative kernel runs whole checkerboard
// sweeps (Fig. 1, Sec. 4.1).  Each CTA owns a contiguous tile of time steps;
// per sweep the even sites move, then the odd sites, then each free parameter
// in order, then statistics, step adaptation and annealing (Sec. 4.1-4.2).
//
// A parameter move (Sec. 4.3) needs the whole path: every CTA evaluates the
// map at the proposed p for its sites into the inactive half of the
// double-buffered cache and a partial change of action, summed exactly (integer
// chunks, see "exact sums" below); after one grid barrier every CTA reads the
// same total and takes the same accept decision, so no second launch or
// broadcast is needed.  In FP32 the HH map of a parameter move runs on packed
// f32x2 arithmetic: two adjacent sites a thread in the general form, the two
// speculative outcomes of a site in the resident form.
//
// Two forms of the site phases:
//  * resident (tiles of at most NT - 32 sites): thread 32 + i owns site
//    n0 + i for the whole launch and keeps its operands in registers; the
//    tile's neighbours are exchanged through shared memory and the two halo
//    sites through global memory, ordered by epoch flags between neighbouring
//    CTAs instead of grid barriers.  Warp 0 draws, reduces, synchronises and
//    decides; while it waits for the other CTAs, the site threads evaluate the
//    next parameter move's map for both outcomes of the pending decision.
//  * general (any tile): threads stride over the tile, operands are read from
//    global memory (L2); in a chain's own launch each site phase ends with a
//    CTA barrier and the neighbours' epoch flags, in a batched launch of
//    split chains with a barrier of the chain's CTAs.
// All waits are bounded in time.
#include <cuda/atomic>
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "scheme.cuh"
#include "stats.cuh"

namespace pimc {

// An exact sum of parameter-move terms (see "exact sums" below).
struct Fix3 {
    long long c[3];
    unsigned long long flags;
};

constexpr long long kFixMask = (1ll << 42) - 1;

template <class R, int NT> struct SweepShared {
    double p[kMaxP], lo[kMaxP], hi[kMaxP], sigp[kMaxP];
    double beta;
    long long sweep, J;
    unsigned fidx, free_mask, nred;
    unsigned accp_win[kMaxP];
    unsigned long long par_acc[kMaxP], par_prop[kMaxP];
    double pnew[kMaxP], elog[kMaxP];  // this sweep's proposal and -log u per parameter
    int inbox[kMaxP];
    R q_cur[kMaxP];                   // current model parameters in R
    R q_new[kMaxP][kMaxP];            // proposed vector for each parameter move, in R
    R halo[kMaxD];                  // trapezoid: F(x_{n1}, p') of the next tile's first site
    R xs[kMaxD][NT];                // resident form: x of site n0 + i at [a][i]
    R gs[kMaxD][NT];                // resident form: cached value of site n0 + i at [a][i]
    Fix3 wfix[NT / 32];             // warp sums of a parameter move's exact CTA sum
    Fix3 cta_fix;                   // CTA sum of a parameter move (CTA-local chains)
    Fix3 wspec[2][NT / 32];         // resident form: site warps' sums of the next move's terms (accept, reject)
    Fix3 cta_spec[2][2];            // resident form: [buffer][accept, reject] CTA sums of the next move's terms
    unsigned long long ep0;         // resident form: epoch base of the neighbour flags
    unsigned bar_phase;             // top bit of the grid-barrier word before the next barrier
    int abort;
    int last_acc;                   // outcome of the latest parameter decision
    unsigned long long site_acc[2], site_prop[2], nonfinite;
    long long tr_n;
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void wait_expired(const Ctx& c)
{
    atomicOr(&c.st->status, kStatusTimeout);
    atomicExch(&c.st->abort, 1);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Barrier of the G CTAs that share a chain (the whole grid of a chain's own
// launch, or a group of a batched launch) on the chain's 32-bit word: every
// CTA adds 1, except rank 0 which adds 2^31 - (G - 1), so the word's top bit
// flips exactly when all G CTAs have arrived and its low bits return to their
// old value.  Arrival is a release (fence, then a relaxed add that returns
// nothing); each CTA knows the top bit before the barrier (`phase`, read at
// the chain's start and toggled at every barrier) and polls with acquire loads
// until it flips.  The wait is bounded by c.wait_ns: on expiry the CTA flags
// kStatusTimeout and the abort word, and every CTA leaves at its next wait.
__device__ __forceinline__ void grid_arrive(const Ctx& c, int rank, int size)
{
    const unsigned add = (rank == 0) ? (0x80000000u - (unsigned)(size - 1)) : 1u;
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    if (rank != c.skip_cta)
        asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(c.bar), "r"(add) : "memory");
}

__device__ __forceinline__ bool grid_wait(const Ctx& c, unsigned phase)
{
    bool ok = true;
    unsigned spins = 0;
    const unsigned long long t0 = global_ns();
    while ((ld_acquire_u32(c.bar) >> 31) == phase) {
        if ((++spins & 63u) == 0u) {
            if (*(volatile int*)&c.st->abort) { ok = false; break; }
            if ((long long)(global_ns() - t0) > c.wait_ns) { wait_expired(c); ok = false; break; }
            if (spins > 4096u) __nanosleep(64);
        }
    }
    return ok;
}

// One thread: arrive, wait, and toggle the tracked top bit.
__device__ __forceinline__ bool grid_sync_one(const Ctx& c, unsigned* phase, int rank, int size)
{
    grid_arrive(c, rank, size);
    const bool ok = grid_wait(c, *phase);
    *phase ^= 1u;
    return ok;
}

// Whole-CTA form.  Returns false when leaving.
__device__ bool grid_barrier(const Ctx& c, int* s_abort, unsigned* phase, int rank, int size)
{
    __syncthreads();
    if (threadIdx.x == 0) *s_abort = !grid_sync_one(c, phase, rank, size);
    __syncthreads();
    return !*s_abort;
}

// Epoch flags between neighbouring CTAs (resident form).  After its sites of
// parity ph have moved in the sweep with epoch e, a CTA stores e into
// flags[ph][b] with a release store (after a CTA barrier, so it publishes the
// CTA's writes); a neighbour polls, bounded, with acquire loads until the flag
// reaches e.  Epochs only grow over a handle's launches (the host passes the
// base in c.ep0).
__device__ __forceinline__ void flag_post(const Ctx& c, int ph, unsigned long long e)
{
    if ((int)blockIdx.x == c.skip_cta) return;
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(c.flags + ph * kMaxGrid + blockIdx.x), "l"(e)
                 : "memory");
}

__device__ __forceinline__ bool flag_wait(const Ctx& c, int ph, int b, unsigned long long e)
{
    bool ok = true;
    unsigned spins = 0;
    const unsigned long long t0 = global_ns();
    const unsigned long long* f = c.flags + ph * kMaxGrid + b;
    while (ld_acquire_u64(f) < e) {
        if ((++spins & 63u) == 0u) {
            if (*(volatile int*)&c.st->abort) { ok = false; break; }
            if ((long long)(global_ns() - t0) > c.wait_ns) { wait_expired(c); ok = false; break; }
            if (spins > 4096u) __nanosleep(64);
        }
    }
    return ok;
}

// ---- checked builds (PIMC_CHECK): site-visit counters and index checks ----
// A site visit of the even phase (kind 0), the odd phase (1) or a parameter
// move's cache write (2) is counted per site; a test compares the counts with
// the number of phases and moves (every site exactly once per phase).  An
// index outside [0, M] sets kStatusBounds and the access is skipped.
#ifdef PIMC_CHECK
__device__ __forceinline__ bool chk_site(const Ctx& c, int kind, int64_t n)
{
    if (n < 0 || n > c.M) {
        atomicOr(&c.st->status, kStatusBounds);
        return false;
    }
    atomicAdd(c.chk + (int64_t)kind * c.ldx + n, 1u);
    return true;
}
__device__ __forceinline__ void chk_move(const Ctx& c)
{
    atomicAdd((unsigned long long*)(c.chk + 3 * c.ldx), 1ull);
}
#else
__device__ __forceinline__ constexpr bool chk_site(const Ctx&, int, int64_t) { return true; }
__device__ __forceinline__ void chk_move(const Ctx&) {}
#endif

int checked_build()
{
#ifdef PIMC_CHECK
    return 1;
#else
    return 0;
#endif
}

// Neighbourhood of site n loaded before its map is evaluated.
template <class R, int D> struct Nbhd {
    R yn, xprev[D], gprev[D], gcur[D], xn1[D], gn1[D];
};

template <class Model, class R>
__device__ __forceinline__ void load_nbhd(const Ctx& c, int64_t n, const R* Fc, Nbhd<R, Model::D>& nb)
{
    constexpr int D = Model::D;
    const R* X = (const R*)c.X;
    const bool trap = c.scheme != kSchemeRK4;
    if (n >= 1) {
        nb.yn = ((const R*)c.y)[n];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            nb.gprev[a] = Fc[a * c.ldf + n - 1];
            nb.xprev[a] = trap ? X[a * c.ldx + n - 1] : R(0);
        }
    }
#pragma unroll
    for (int a = 0; a < D; ++a) nb.gcur[a] = (n < cache_len(c)) ? Fc[a * c.ldf + n] : R(0);
    if (n < c.M) {
#pragma unroll
        for (int a = 0; a < D; ++a) {
            nb.xn1[a] = X[a * c.ldx + n + 1];
            nb.gn1[a] = trap ? Fc[a * c.ldf + n + 1] : R(0);
        }
    }
}

// Local change of action for x_n -> xp with cached value gp (Fig. 1 steps
// (c)-(g)): the measurement term at n (n >= 1) and the model-error terms
// eps_n (n >= 1) and eps_{n+1} (n <= M-1), each as 1/2 R (e' - e)(e' + e).
template <class Model, class R>
__device__ __forceinline__ R site_delta(const Ctx& c, const Coef<R>& k, int64_t n, const R* x, const R* xp,
                                        const R* gp, R beta, const Nbhd<R, Model::D>& nb)
{
    constexpr int D = Model::D;
    R dA = R(0);
    if (n >= 1) {
        dA += sqdiff<R>(k.Rm, xp[0] - nb.yn, x[0] - nb.yn);
        R dAf = R(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const R e = eps_of<R>(c, k, nb.xprev[a], x[a], nb.gprev[a], nb.gcur[a]);
            const R ep = eps_of<R>(c, k, nb.xprev[a], xp[a], nb.gprev[a], gp[a]);
            dAf += sqdiff<R>(k.Rf[a], ep, e);
        }
        dA += beta * dAf;
    }
    if (n < c.M) {
        R dAf = R(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const R e = eps_of<R>(c, k, x[a], nb.xn1[a], nb.gcur[a], nb.gn1[a]);
            const R ep = eps_of<R>(c, k, xp[a], nb.xn1[a], gp[a], nb.gn1[a]);
            dAf += sqdiff<R>(k.Rf[a], ep, e);
        }
        dA += beta * dAf;
    }
    return dA;
}

// Proposal increments of site n at sweep s: D Box-Muller normals (cos then
// sin per pair of blocks 0, 1) or U(-1, 1) from the same words, and the
// accept uniform (block 2).
template <class Model, class R>
__device__ __forceinline__ void site_draws(const Ctx& c, long long s, int64_t n, R* z, R& u)
{
    constexpr int D = Model::D;
#pragma unroll
    for (int pair = 0; 2 * pair < D; ++pair) {
        R z0, z1;
        const uint4 w = draw_block(c.seed, c.chain, (uint64_t)s, (uint32_t)n, kKindSite, pair);
        if (c.proposal == kProposalUniform) {
            z0 = R(2) * Num<R>::uni(w.x, w.y) - R(1);
            z1 = R(2) * Num<R>::uni(w.z, w.w) - R(1);
        } else {
            Num<R>::box_muller(w, z0, z1);
        }
        z[2 * pair] = z0;
        if (2 * pair + 1 < D) z[2 * pair + 1] = z1;
    }
    const uint4 w = draw_block(c.seed, c.chain, (uint64_t)s, (uint32_t)n, kKindSite, 2u);
    u = Num<R>::uni(w.x, w.y);
}

// The draws of site n's move at sweep s: the proposal increments z and
// E = -log u of the accept uniform.
template <class Model, class R>
__device__ __forceinline__ void site_draw(const Ctx& c, long long s, int64_t n, R* z, R& E)
{
    R u;
    site_draws<Model, R>(c, s, n, z, u);
    E = neglog<R>(u);
}

// The proposal from its increments: x' = x + sigma z (one fma a component)
// and its cached value.
template <class Model, class R>
__device__ __forceinline__ void site_propose_from(const Ctx& c, const Coef<R>& k, int64_t n, const R* pr,
                                                  const R* x, const R* sg, R drive, const R* z, R* xp, R* gp)
{
    constexpr int D = Model::D;
#pragma unroll
    for (int a = 0; a < D; ++a) xp[a] = fma(sg[a], z[a], x[a]);
    if (n < cache_len(c)) cache_value_at<Model, R>(c, k, xp, pr, drive, gp);
    else {
#pragma unroll
        for (int a = 0; a < D; ++a) gp[a] = R(0);
    }
}

// A site move from operands in registers, in two halves.  The proposal:
// x' = x + sigma z, its cached value, and -log u of the accept uniform.
template <class Model, class R>
__device__ __forceinline__ void site_propose(const Ctx& c, const Coef<R>& k, int64_t n, long long s, const R* pr,
                                             const R* x, const R* sg, R drive, R* xp, R* gp, R& E)
{
    constexpr int D = Model::D;
    R z[D];
    site_draw<Model, R>(c, s, n, z, E);
    site_propose_from<Model, R>(c, k, n, pr, x, sg, drive, z, xp, gp);
}

// The decision: Delta A_n and the Metropolis rule written as dA < -log u
// (Eq. (Paccept); NaN compares false).
template <class Model, class R>
__device__ __forceinline__ bool site_decide(const Ctx& c, const Coef<R>& k, int64_t n, const R* x, const R* xp,
                                            const R* gp, R beta, R E, const Nbhd<R, Model::D>& nb,
                                            unsigned long long& nonfinite)
{
    const R dA = site_delta<Model, R>(c, k, n, x, xp, gp, beta, nb);
    if (!isfinite(dA)) ++nonfinite;
    return dA < E;
}

template <class Model, class R>
__device__ __forceinline__ bool site_core(const Ctx& c, const Coef<R>& k, int64_t n, long long s, const R* pr,
                                          R beta, const R* x, const R* sg, R drive, const Nbhd<R, Model::D>& nb,
                                          R* xp, R* gp, unsigned long long& nonfinite)
{
    R E;
    site_propose<Model, R>(c, k, n, s, pr, x, sg, drive, xp, gp, E);
    return site_decide<Model, R>(c, k, n, x, xp, gp, beta, E, nb, nonfinite);
}

// General form of a site move: operands from global memory, store on accept.
template <class Model, class R>
__device__ __forceinline__ bool site_move(const Ctx& c, const Coef<R>& k, int64_t n, long long s, const R* pr,
                                          R beta, R* Fc, unsigned long long& nonfinite)
{
    constexpr int D = Model::D;
    R* X = (R*)c.X;
    const R* sig = (const R*)c.sig;
    R x[D], sg[D], xp[D], gp[D];
    Nbhd<R, D> nb;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        x[a] = X[a * c.ldx + n];
        sg[a] = sig[a * c.ldx + n];
    }
    load_nbhd<Model, R>(c, n, Fc, nb);
    const bool cached = n < cache_len(c);
    const R drive = cached ? ((const R*)c.I)[drive_index(c, n)] : R(0);
    const bool acc = site_core<Model, R>(c, k, n, s, pr, beta, x, sg, drive, nb, xp, gp, nonfinite);
    if (acc) {
#pragma unroll
        for (int a = 0; a < D; ++a) X[a * c.ldx + n] = xp[a];
        if (cached) {
#pragma unroll
            for (int a = 0; a < D; ++a) Fc[a * c.ldf + n] = gp[a];
        }
        atomicAdd(&c.acc_win[n], 1u);
    }
    return acc;
}

// RK4 scheme: site n's share of a parameter move -- f(x_n, p') into the
// inactive cache and beta/2 sum_a Rf_a [(x_{n+1} - f')^2 - (x_{n+1} - f)^2].
template <class Model, class R>
__device__ __forceinline__ R param_term(const Ctx& c, const Coef<R>& k, int64_t n, const R* pq, R beta,
                                        const R* Fc, R* Fn)
{
    constexpr int D = Model::D;
    const R* X = (const R*)c.X;
    R x[D], fp[D], xn1[D], fc[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        x[a] = X[a * c.ldx + n];
        xn1[a] = X[a * c.ldx + n + 1];
        fc[a] = Fc[a * c.ldf + n];
    }
    rk4_map<Model, R>(x, pq, ((const R*)c.I)[n], k.dt, fp);
#pragma unroll
    for (int a = 0; a < D; ++a) Fn[a * c.ldf + n] = fp[a];
    if constexpr (std::is_same<R, float>::value) {
        return rk4_term_lanes<float, D>(beta, k.Rf, xn1, fp, fc);
    } else {
        R t = R(0);
#pragma unroll
        for (int a = 0; a < D; ++a) t += beta * sqdiff<R>(k.Rf[a], xn1[a] - fp[a], xn1[a] - fc[a]);
        return t;
    }
}

// Trapezoid scheme, first pass: F(x_n, p') of site n into the inactive cache.
template <class Model, class R>
__device__ __forceinline__ void trap_field(const Ctx& c, const Coef<R>& k, int64_t n, const R* pq, R* Fn, R* g)
{
    constexpr int D = Model::D;
    const R* X = (const R*)c.X;
    R x[D];
#pragma unroll
    for (int a = 0; a < D; ++a) x[a] = X[a * c.ldx + n];
    cache_value<Model, R>(c, k, x, pq, n, g);
    if (Fn) {
#pragma unroll
        for (int a = 0; a < D; ++a) Fn[a * c.ldf + n] = g[a];
    }
}

// Trapezoid scheme, second pass: the change of eps_{n+1} when F_n, F_{n+1}
// become F'_n, F'_{n+1} (gn1p: the new field at n+1).
template <class Model, class R>
__device__ __forceinline__ R trap_term(const Ctx& c, const Coef<R>& k, int64_t n, R beta, const R* Fc, const R* Fn,
                                       const R* gn1p)
{
    constexpr int D = Model::D;
    const R* X = (const R*)c.X;
    R t = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const R xn = X[a * c.ldx + n], xn1 = X[a * c.ldx + n + 1];
        const R e = eps_of<R>(c, k, xn, xn1, Fc[a * c.ldf + n], Fc[a * c.ldf + n + 1]);
        const R ep = eps_of<R>(c, k, xn, xn1, Fn[a * c.ldf + n], gn1p[a]);
        t += beta * sqdiff<R>(k.Rf[a], ep, e);
    }
    return t;
}

// ---- exact sums of parameter-move terms ---------------------------------------
// A term t enters as the integer T = t 2^64 truncated toward zero (|t| < 2^62;
// terms below 2^-64 vanish), held in three signed 64-bit chunks of 42 bits,
// T = c0 + c1 2^42 + c2 2^84.  Chunk-wise integer additions of up to 2^21
// terms neither overflow nor round, so the change of action of a parameter
// move is summed exactly and in no particular order: every CTA, tiling and
// form obtains the same bits, and the result, rounded once to FP64, is at
// least as accurate as an FP64 summation.  Infinite terms (|t| >= 2^62) and
// NaN set flags (1: +inf, 2: -inf, 4: NaN) that make the total +-inf or NaN.
// (struct Fix3: see "exact sums of parameter-move terms" below)

__device__ __forceinline__ void fix_zero(Fix3& f)
{
    f.c[0] = f.c[1] = f.c[2] = 0;
    f.flags = 0ull;
}

// Adds sign * m 2^e2 for an integer m < 2^53: T = m 2^(e2 + 64) as a 128-bit
// integer (hi:lo), cut into the three chunks.
__device__ __forceinline__ void fix_add_parts(Fix3& f, unsigned long long m, int e2, bool neg)
{
    const int sh = e2 + 64;  // bit of T that m's bit 0 lands on
    if (m != 0ull && sh + (64 - __clzll((long long)m)) > 126) {
        f.flags |= neg ? 2ull : 1ull;
        return;
    }
    unsigned long long lo = 0ull, hi = 0ull;
    if (sh >= 64) hi = m << (sh - 64);
    else if (sh > 0) { lo = m << sh; hi = m >> (64 - sh); }
    else if (sh > -64) lo = m >> (-sh);
    const unsigned long long k = (unsigned long long)kFixMask;
    long long c0 = (long long)(lo & k), c1 = (long long)(((lo >> 42) | (hi << 22)) & k), c2 = (long long)(hi >> 20);
    if (neg) {
        c0 = -c0;
        c1 = -c1;
        c2 = -c2;
    }
    f.c[0] += c0;
    f.c[1] += c1;
    f.c[2] += c2;
}

__device__ __forceinline__ void fix_add(Fix3& f, float t)
{
    const unsigned b = __float_as_uint(t);
    const unsigned ex = (b >> 23) & 0xffu, man = b & 0x7fffffu;
    const bool neg = (b >> 31) != 0u;
    if (ex == 0xffu) f.flags |= man ? 4ull : (neg ? 2ull : 1ull);
    else if (ex == 0u) fix_add_parts(f, man, -149, neg);
    else fix_add_parts(f, man | 0x800000u, (int)ex - 150, neg);
}

__device__ __forceinline__ void fix_add(Fix3& f, double t)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(t);
    const int ex = (int)((b >> 52) & 0x7ffull);
    const unsigned long long man = b & ((1ull << 52) - 1ull);
    const bool neg = (b >> 63) != 0ull;
    if (ex == 0x7ff) f.flags |= man ? 4ull : (neg ? 2ull : 1ull);
    else if (ex == 0) fix_add_parts(f, man, -1074, neg);
    else fix_add_parts(f, man | (1ull << 52), ex - 1075, neg);
}

__device__ __forceinline__ void fix_normalize(Fix3& f)
{
    f.c[1] += f.c[0] >> 42;
    f.c[0] &= kFixMask;
    f.c[2] += f.c[1] >> 42;
    f.c[1] &= kFixMask;
}

// The sum as a double: carries normalised (c0, c1 in [0, 2^42), the sign in
// c2), the magnitude formed from non-negative chunks added from the low one up
// (two roundings at most, no cancellation), then the sign.
__device__ __forceinline__ double fix_value(Fix3 f)
{
    if (f.flags) {
        if ((f.flags & 4ull) || (f.flags & 3ull) == 3ull) return __longlong_as_double(0x7ff8000000000000ll);
        return __longlong_as_double((f.flags & 1ull) ? 0x7ff0000000000000ll : (long long)0xfff0000000000000ull);
    }
    fix_normalize(f);
    const bool neg = f.c[2] < 0;
    if (neg) {
#pragma unroll
        for (int j = 0; j < 3; ++j) f.c[j] = -f.c[j];
        fix_normalize(f);
    }
    const double mag = fma((double)f.c[2], 0x1p20, fma((double)f.c[1], 0x1p-22, (double)f.c[0] * 0x1p-64));
    return neg ? -mag : mag;
}

// Whether the exact sum s is below e: Eq. (Paccept) as dA < -log u, decided
// in the fixed point (e truncated like the terms; -log u is a multiple of
// 2^-64 whenever u < 0.9997).  A NaN or +inf sum rejects, -inf accepts.
__device__ __forceinline__ bool fix_less(Fix3 s, double e)
{
    if (s.flags) return s.flags == 2ull;
    Fix3 t;
    fix_zero(t);
    fix_add(t, e);
    if (t.flags) return t.flags == 1ull;
    fix_normalize(s);
    fix_normalize(t);
    if (s.c[2] != t.c[2]) return s.c[2] < t.c[2];
    if (s.c[1] != t.c[1]) return s.c[1] < t.c[1];
    return s.c[0] < t.c[0];
}

// A thread's running exact sum of FP32 terms, for loops over many sites: the
// same integer T = t 2^64 truncated toward zero as fix_add, kept as one
// 128-bit two's complement integer (hi:lo) -- a shift and a 128-bit add or
// subtract a term instead of a split into three chunks.  Terms of magnitude
// 2^36 or more, and non-finite ones, go to the Fix3 sum instead, so up to 2^26
// terms cannot overflow; acc_fold adds the 128-bit sum into the Fix3 sum.  The
// total is the same integer either way, so every form keeps the same bits.
struct Acc128 {
    unsigned long long lo, hi;
};

__device__ __forceinline__ void acc_add(Acc128& a, Fix3& big, float t)
{
    const unsigned b = __float_as_uint(t);
    const unsigned ex = (b >> 23) & 0xffu;
    if (ex >= 127u + 36u) {
        fix_add(big, t);
        return;
    }
    const unsigned long long man = ex ? (unsigned long long)((b & 0x7fffffu) | 0x800000u) : (unsigned long long)(b & 0x7fffffu);
    const int sh = (ex ? (int)ex - 150 : -149) + 64;  // bit of T that man's bit 0 lands on (<= 77)
    unsigned long long lo = 0ull, hi = 0ull;
    if (sh >= 64) hi = man << (sh - 64);
    else if (sh > 40) { lo = man << sh; hi = man >> (64 - sh); }
    else if (sh >= 0) lo = man << sh;
    else if (sh > -24) lo = man >> (-sh);
    if (b >> 31) {
        const unsigned long long l2 = a.lo - lo;
        a.hi = a.hi - hi - (a.lo < lo ? 1ull : 0ull);
        a.lo = l2;
    } else {
        const unsigned long long l2 = a.lo + lo;
        a.hi = a.hi + hi + (l2 < lo ? 1ull : 0ull);
        a.lo = l2;
    }
}

__device__ __forceinline__ void acc_fold(const Acc128& a, Fix3& f)
{
    f.c[0] += (long long)(a.lo & (unsigned long long)kFixMask);
    f.c[1] += (long long)(((a.lo >> 42) | (a.hi << 22)) & (unsigned long long)kFixMask);
    f.c[2] += (long long)a.hi >> 20;
}

// Warp sum of Fix3 values, valid in every lane.  Each lane's value is
// normalised (c0, c1 in [0, 2^42)) and cut into 21-bit pieces -- the top
// chunk's upper piece signed -- whose 32-lane sums fit 32-bit integers, so the
// warp adds them with seven independent redux.sync reductions instead of
// five dependent rounds of 64-bit shuffles.  A top chunk of 2^41 or more
// (terms near the 2^62 limit) sends the warp to the shuffle rounds.
__device__ __forceinline__ Fix3 fix_warp_sum(Fix3 f)
{
    constexpr unsigned kAll = 0xffffffffu;
    fix_normalize(f);
    const long long lim = 1ll << 41;
    if (__any_sync(kAll, f.c[2] >= lim || f.c[2] < -lim)) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) f.c[j] += __shfl_xor_sync(kAll, f.c[j], off);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) f.flags |= __shfl_xor_sync(kAll, f.flags, off);
        return f;
    }
    const unsigned m21 = (1u << 21) - 1u;
    const unsigned s0 = __reduce_add_sync(kAll, (unsigned)f.c[0] & m21);
    const unsigned s1 = __reduce_add_sync(kAll, (unsigned)(f.c[0] >> 21));
    const unsigned s2 = __reduce_add_sync(kAll, (unsigned)f.c[1] & m21);
    const unsigned s3 = __reduce_add_sync(kAll, (unsigned)(f.c[1] >> 21));
    const unsigned s4 = __reduce_add_sync(kAll, (unsigned)f.c[2] & m21);
    const int s5 = __reduce_add_sync(kAll, (int)(f.c[2] >> 21));
    Fix3 r;
    r.c[0] = (long long)s0 + (long long)s1 * (1ll << 21);
    r.c[1] = (long long)s2 + (long long)s3 * (1ll << 21);
    r.c[2] = (long long)s4 + (long long)s5 * (1ll << 21);
    r.flags = __reduce_or_sync(kAll, (unsigned)f.flags);
    return r;
}

// CTA sum of every thread's Fix3 (one CTA barrier inside), carries
// normalised; valid in thread 0.
template <int NT>
__device__ __forceinline__ Fix3 fix_cta_sum(Fix3 f, Fix3* wfix)
{
    f = fix_warp_sum(f);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wfix[w] = f;
    __syncthreads();
    Fix3 t;
    fix_zero(t);
    if (threadIdx.x < 32) {
        if (lane < NT / 32) t = wfix[lane];
        t = fix_warp_sum(t);
        fix_normalize(t);
    }
    return t;
}

// Synchronisation policies of a chain's sweep.  GridSync: the chain is tiled
// over `size` CTAs -- all CTAs of a cooperative launch, or a group of a
// batched launch -- the CTA of rank r owning tile r (barriers on the chain's
// word; each CTA adds its exact partial into a slot of three integer
// accumulators before the barrier of a parameter move and reads the total
// after it).  BlockSync: one CTA owns the whole chain (CTA barriers, the CTA
// sum is the total).  Both give the same bits for the same chain.  Slots
// rotate over three (a slot is cleared by rank 0 one move after its use, when
// every CTA has read it; all are cleared before each launch).
struct GridSync {
    int rank, size;
    // general form: order the site phases by the neighbours' epoch flags
    // instead of grid barriers (a chain's own launch; c.ep0 is its epoch base)
    int site_flags = 0;
    static constexpr bool tiled = true;
    __device__ __forceinline__ bool barrier(const Ctx& c, int* s_abort, unsigned* phase) const
    {
        return grid_barrier(c, s_abort, phase, rank, size);
    }
    __device__ __forceinline__ bool arrive_wait(const Ctx& c, unsigned* phase) const
    {
        return grid_sync_one(c, phase, rank, size);
    }
    // thread 0, before the barrier
    __device__ __forceinline__ void publish(const Ctx& c, unsigned slot, const Fix3& f, Fix3*) const
    {
        unsigned long long* acc = (unsigned long long*)c.partials + 4 * slot;
#pragma unroll
        for (int j = 0; j < 3; ++j)
            asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(acc + j), "l"((unsigned long long)f.c[j])
                         : "memory");
        if (f.flags) asm volatile("red.relaxed.gpu.global.or.b64 [%0], %1;" ::"l"(acc + 3), "l"(f.flags) : "memory");
    }
    // thread 0, after the barrier
    __device__ __forceinline__ Fix3 total(const Ctx& c, unsigned slot, const Fix3*) const
    {
        const unsigned long long* acc = (const unsigned long long*)c.partials + 4 * slot;
        Fix3 t;
#pragma unroll
        for (int j = 0; j < 3; ++j) t.c[j] = (long long)__ldcg(acc + j);
        t.flags = __ldcg(acc + 3);
        return t;
    }
    // thread 0, after reading the total of `slot`: clear the previous slot
    __device__ __forceinline__ void recycle(const Ctx& c, unsigned slot) const
    {
        if (rank != 0) return;
        unsigned long long* acc = (unsigned long long*)c.partials + 4 * ((slot + 2u) % 3u);
#pragma unroll
        for (int j = 0; j < 4; ++j) __stcg(acc + j, 0ull);
    }
    __device__ __forceinline__ bool lead() const { return rank == 0; }
};

struct BlockSync {
    static constexpr bool tiled = false;
    int site_flags = 0;
    __device__ __forceinline__ bool barrier(const Ctx&, int*, unsigned*) const
    {
        __syncthreads();
        return true;
    }
    __device__ __forceinline__ bool arrive_wait(const Ctx&, unsigned*) const { return true; }
    __device__ __forceinline__ void publish(const Ctx&, unsigned, const Fix3& f, Fix3* cta) const { *cta = f; }
    __device__ __forceinline__ Fix3 total(const Ctx&, unsigned, const Fix3* cta) const { return *cta; }
    __device__ __forceinline__ void recycle(const Ctx&, unsigned) const {}
    __device__ __forceinline__ bool lead() const { return true; }
};

// ---- pieces shared by both forms --------------------------------------------

template <class Model, class R, int NT>
__device__ __forceinline__ void load_chain_state(const Ctx& c, SweepShared<R, NT>& sh)
{
    const DevState* g = c.st;
    for (int l = 0; l < kMaxP; ++l) {
        sh.p[l] = g->p[l]; sh.lo[l] = g->lo[l]; sh.hi[l] = g->hi[l]; sh.sigp[l] = g->sigp[l];
        sh.accp_win[l] = g->accp_win[l]; sh.par_acc[l] = g->par_acc[l]; sh.par_prop[l] = g->par_prop[l];
    }
    sh.beta = g->beta; sh.sweep = g->sweep; sh.J = g->J; sh.fidx = g->fidx;
    sh.free_mask = g->free_mask; sh.nred = 0; sh.abort = 0; sh.tr_n = g->tr_n; sh.last_acc = 0;
    sh.site_acc[0] = sh.site_acc[1] = sh.site_prop[0] = sh.site_prop[1] = sh.nonfinite = 0ull;
    sh.ep0 = c.ep0;
    sh.bar_phase = c.bar ? (*(volatile const unsigned*)c.bar) >> 31 : 0u;
    Model::prep(sh.p, sh.q_cur);
}

// The parameter-move draws of sweep s, parameter l (Philox kind 1): the
// proposal increment z (Box-Muller normal, or U(-1, 1)) and -log u of the
// accept uniform.
__device__ __forceinline__ void param_draw(const Ctx& c, long long s, int l, double& z, double& elog)
{
    double z1;
    const uint4 wz = draw_block(c.seed, c.chain, (uint64_t)s, (uint32_t)l, kKindParam, 0u);
    if (c.proposal == kProposalUniform) z = 2.0 * u01d(wz.x, wz.y) - 1.0;
    else Num<double>::box_muller(wz, z, z1);
    const uint4 w = draw_block(c.seed, c.chain, (uint64_t)s, (uint32_t)l, kKindParam, 1u);
    elog = -log(u01d(w.x, w.y));
}

// This sweep's proposal for parameter l (one thread per parameter) from its
// draws.  p_l changes only in its own move, so p'_l = p_l + sigma_l z_l is
// fixed at the sweep's start; the proposed vector of move l is completed after
// the earlier moves from q_new[l] (components l, and 7 with l = 6).
template <class Model, class R, int NT>
__device__ __forceinline__ void set_param_proposal(SweepShared<R, NT>& sh, int l, double z, double elog)
{
    const double pl = sh.p[l] + sh.sigp[l] * z;
    sh.pnew[l] = pl;
    sh.elog[l] = elog;
    sh.inbox[l] = (pl >= sh.lo[l] && pl <= sh.hi[l]) ? 1 : 0;
    double pv[kMaxP];
#pragma unroll
    for (int q = 0; q < kMaxP; ++q) pv[q] = (q == l) ? pl : sh.p[q];
    Model::prep(pv, sh.q_new[l]);
}

template <class Model, class R, int NT>
__device__ __forceinline__ void draw_param_proposal(const Ctx& c, SweepShared<R, NT>& sh, long long s, int l)
{
    if (!((sh.free_mask >> l) & 1u)) return;
    double z, elog;
    param_draw(c, s, l, z, elog);
    set_param_proposal<Model, R, NT>(sh, l, z, elog);
}

// The model-parameter vector of move l applied to q (components l, and 7
// with l = 6).  Static indices keep q in registers.
template <class R, int NT>
__device__ __forceinline__ void apply_move(R* q, const SweepShared<R, NT>& sh, int l)
{
#pragma unroll
    for (int j = 0; j < kMaxP; ++j)
        if (j == l || (j == 7 && l == 6)) q[j] = sh.q_new[l][j];
}

// Decision of move l on the exact total change of action: Eq. (Paccept) as
// dA < -log u (fix_less).  One thread.
template <class R, int NT>
__device__ __forceinline__ void decide(SweepShared<R, NT>& sh, int l, const Fix3& v)
{
    const int acc = fix_less(v, sh.elog[l]) ? 1 : 0;
    if (acc) {
        sh.p[l] = sh.pnew[l];
        sh.q_cur[l] = sh.q_new[l][l];
        if (l == 6) sh.q_cur[7] = sh.q_new[l][7];
        sh.fidx ^= 1u;
        sh.accp_win[l] += 1u;
        sh.par_acc[l] += 1ull;
    }
    sh.last_acc = acc;
    sh.nred += 1u;
}

// Step adaptation of the parameters during burn-in (Sec. 4.2).  One thread.
template <int NP, class R, int NT>
__device__ __forceinline__ void adapt_params(const Ctx& c, SweepShared<R, NT>& sh)
{
    for (int l = 0; l < NP; ++l) {
        if ((sh.free_mask >> l) & 1u)
            sh.sigp[l] *= 1.0 + c.alpha * ((double)sh.accp_win[l] / (double)c.n_skip - c.f_acc);
        sh.accp_win[l] = 0u;
    }
}

// End of a sweep: parameter trace, annealing (Eq. (fbeta)), counters.
template <int NP, class R, int NT, class Sync>
__device__ __forceinline__ void end_sweep(const Ctx& c, SweepShared<R, NT>& sh, long long s, bool record,
                                          const Sync& sync)
{
    const int tid = threadIdx.x;
    if (c.trace && sync.lead() && tid < NP) c.trace[(sh.tr_n % c.trace_cap) * NP + tid] = sh.p[tid];
    __syncthreads();
    if (tid == 0) {
        sh.beta = (s + 1 < c.n_cool) ? sh.beta * c.fbeta : 1.0;
        sh.sweep = s + 1;
        if (record) sh.J += 1;
        if (c.trace) sh.tr_n += 1;
    }
    __syncthreads();
}

// Adds this CTA's counters and (lead CTA) writes the chain state back.
template <class R, int NT, class Sync>
__device__ __forceinline__ void store_chain_state(const Ctx& c, SweepShared<R, NT>& sh, const Sync& sync,
                                                  const unsigned long long* acc, const unsigned long long* prop,
                                                  unsigned long long nf)
{
    __syncthreads();
    atomicAdd(&sh.site_acc[0], acc[0]);
    atomicAdd(&sh.site_acc[1], acc[1]);
    atomicAdd(&sh.site_prop[0], prop[0]);
    atomicAdd(&sh.site_prop[1], prop[1]);
    atomicAdd(&sh.nonfinite, nf);
    __syncthreads();
    if (threadIdx.x == 0) {
        DevState* g = c.st;
        atomicAdd(&g->site_acc[0], sh.site_acc[0]);
        atomicAdd(&g->site_acc[1], sh.site_acc[1]);
        atomicAdd(&g->site_prop[0], sh.site_prop[0]);
        atomicAdd(&g->site_prop[1], sh.site_prop[1]);
        atomicAdd(&g->nonfinite, sh.nonfinite);
        if (sync.lead()) {
            for (int l = 0; l < kMaxP; ++l) {
                g->p[l] = sh.p[l]; g->sigp[l] = sh.sigp[l]; g->accp_win[l] = sh.accp_win[l];
                g->par_acc[l] = sh.par_acc[l]; g->par_prop[l] = sh.par_prop[l];
            }
            g->beta = sh.beta; g->sweep = sh.sweep; g->J = sh.J; g->fidx = sh.fidx; g->tr_n = sh.tr_n;
        }
    }
    __syncthreads();
}

// Shared-memory staging of the paired parameter-move loop: per thread and
// buffer, the operands of one pair (n, n + 1) -- x_n, x_{n+1} (4 float2),
// x_{n+2} (4 floats), the cached f_n, f_{n+1} (4 float2) and the drive
// (float2) -- copied from global memory with cp.async while the thread
// evaluates the pair before, two buffers in turn.  Each thread reads only its
// own slots, so no CTA barrier is needed; the layout is [buffer][field][thread]
// (consecutive threads, consecutive words: no bank conflicts).  It lives in
// the kernel's dynamic shared memory.
template <int NT> struct PairStage {
    float2 x[2][4][NT];
    float2 fc[2][4][NT];
    float2 I[2][NT];
    float xn2[2][4][NT];
};

__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ unsigned dynamic_smem_bytes()
{
    unsigned v;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

// Dynamic shared memory a sweep kernel of this model and arithmetic type is
// launched with (the paired loop's staging; none for the other forms).
template <class Model, class R, int NT> struct StageBytes { static constexpr int value = 0; };
template <int NT> struct StageBytes<HH<float>, float, NT> { static constexpr int value = (int)sizeof(PairStage<NT>); };

// RK4 scheme, FP32 HH: the sites [n0, nend) of a parameter move two at a time,
// (n, n + 1) with n - n0 even, on the packed f32x2 lane form -- per site the
// same bits as param_term.  n0 is even (tiles have even length), so the pair
// copies are 8-byte aligned; an unpaired last site is lane x alone (lane y
// then reads x_{n+1}, f_{n+1}, I_{n+1}, inside the rows, and is dropped).  The
// operands come through the shared-memory staging, the next pair's copies in
// flight while this pair is evaluated; every launch of a kernel that runs this
// loop passes the staging's size (a kernel without it sets kStatusBounds and
// skips the move's terms rather than touch memory it does not have).
template <int NT>
__device__ __forceinline__ void param_terms_paired(const Ctx& c, const Coef<float>& k, int64_t n0, int64_t nend,
                                                   const float* pq, float beta, const float* Fc, float* Fn,
                                                   Fix3& part)
{
    extern __shared__ __align__(16) unsigned char pimc_dyn_smem[];
    if (dynamic_smem_bytes() < sizeof(PairStage<NT>)) {
        if (threadIdx.x == 0) atomicOr(&c.st->status, kStatusBounds);
        return;
    }
    const float* X = (const float*)c.X;
    const float* I = (const float*)c.I;
    const int tid = threadIdx.x;
    float2 q2[kMaxP];
#pragma unroll
    for (int j = 0; j < kMaxP; ++j) q2[j] = splat<float2>(pq[j]);
    const float2 dt2 = splat<float2>(k.dt), beta2 = splat<float2>(beta);
    const float2 hdt2 = splat<float2>(__fmul_rn(0.5f, k.dt)), sdt2 = splat<float2>(__fdiv_rn(k.dt, 6.0f));
    Acc128 acc{0ull, 0ull};
    PairStage<NT>* st = (PairStage<NT>*)pimc_dyn_smem;
    int64_t n = n0 + 2 * (int64_t)tid;
    // the copies of pair (m, m + 1) into buffer b (m < nend)
    auto issue = [&](int b, int64_t m) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            cp_async8(&st->x[b][a][tid], X + a * c.ldx + m);
            cp_async8(&st->fc[b][a][tid], Fc + a * c.ldf + m);
            if (m + 1 < nend) cp_async4(&st->xn2[b][a][tid], X + a * c.ldx + m + 2);
            else st->xn2[b][a][tid] = 0.0f;
        }
        cp_async8(&st->I[b][tid], I + m);
    };
    if (n < nend) issue(0, n);
    cp_async_commit();
    for (int buf = 0; n < nend; n += 2 * NT, buf ^= 1) {
        const bool two = n + 1 < nend;
        if (n + 2 * NT < nend) issue(buf ^ 1, n + 2 * NT);
        cp_async_commit();
        cp_async_wait<1>();  // this pair's group has landed
        float2 x[4], xn1[4], fc[4], fp[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            x[a] = st->x[buf][a][tid];
            xn1[a] = make_float2(x[a].y, st->xn2[buf][a][tid]);
            fc[a] = st->fc[buf][a][tid];
        }
        hh_rk4_lanes<float2>(x, q2, st->I[buf][tid], dt2, hdt2, sdt2, fp);
        if (chk_site(c, 2, n) && (!two || chk_site(c, 2, n + 1))) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                if (two) *(float2*)(Fn + a * c.ldf + n) = fp[a];
                else Fn[a * c.ldf + n] = fp[a].x;
            }
        }
        const float2 t = rk4_term_lanes<float2, 4>(beta2, k.Rf, xn1, fp, fc);
        acc_add(acc, part, t.x);
        if (two) acc_add(acc, part, t.y);
    }
    cp_async_wait<0>();
    acc_fold(acc, part);
}

// ---- general form -----------------------------------------------------------

// n_sweeps checkerboard sweeps of one chain over the sites [n0, n1) this CTA
// owns, threads striding over the tile.
template <class Model, class R, int NT, class Sync>
__device__ void sweep_chain_general(const Ctx& c, int64_t n0, int64_t n1, int64_t n_sweeps, SweepShared<R, NT>& sh,
                                    const Sync& sync)
{
    constexpr int D = Model::D, NP = Model::NP;
    const int tid = threadIdx.x;
    const Coef<R> kc(c);
    const int64_t M = c.M;
    unsigned long long my_acc[2] = {0ull, 0ull}, my_prop[2] = {0ull, 0ull}, my_nf = 0ull;
    R* sig = (R*)c.sig;

    for (int64_t k = 0; k < n_sweeps; ++k) {
        const long long s = sh.sweep;
        const unsigned long long ep = sh.ep0 + (unsigned long long)k + 1ull;
        // proposals by the last warp (idle in the site phases at small M); no
        // barrier here: the CTA barrier that ends the even phase publishes them
        if (tid >= NT - 32 && tid - (NT - 32) < NP) draw_param_proposal<Model, R, NT>(c, sh, s, tid - (NT - 32));
        const R beta = R(sh.beta);
        R pr[kMaxP];
#pragma unroll
        for (int q = 0; q < kMaxP; ++q) pr[q] = sh.q_cur[q];

        // ---- even then odd sites (Sec. 4.1) ----
        // With site flags (tiles of even length, so a tile's first site is
        // even and its last odd): the first site waits for the previous
        // tile's flag of the previous sweep (its last site and cache final;
        // the launch orders the first sweep), the last site for the next
        // tile's even flag of this sweep (its first site moved); nothing else
        // crosses a tile, so a CTA barrier ends each phase.
#pragma unroll
        for (int parity = 0; parity < 2; ++parity) {
            R* Fc = (R*)c.F[sh.fidx];
            const int64_t first = n0 + (((n0 & 1) != parity) ? 1 : 0);
            for (int64_t n = first + 2 * (int64_t)tid; n < n1; n += 2 * NT) {
                if (!chk_site(c, parity, n)) continue;
                if constexpr (Sync::tiled) {
                    if (sync.site_flags) {
                        // the holder's warp waits as one (a lane left behind
                        // would run its site alone after the others)
                        const bool left = parity == 0 && n == n0 && n0 >= 1 && k > 0;
                        const bool right = parity == 1 && n == n1 - 1 && n1 <= M;
                        const unsigned m = __activemask();
                        bool ok = true;
                        if (__any_sync(m, left || right)) {
                            if (left) ok = flag_wait(c, 1, sync.rank - 1, ep - 1ull);
                            if (right) ok = flag_wait(c, 0, sync.rank + 1, ep);
                            if (!ok) sh.abort = 1;
                            __syncwarp(m);
                        }
                        if (!ok) continue;  // leaving: the phase's CTA barrier reads the abort
                    }
                }
                my_acc[parity] += site_move<Model, R>(c, kc, n, s, pr, beta, Fc, my_nf) ? 1ull : 0ull;
                my_prop[parity] += 1ull;
            }
            if (Sync::tiled && sync.site_flags) {
                __syncthreads();
                if (sh.abort) goto done;
                if (parity == 0 && tid == 0) flag_post(c, 0, ep);
            } else if (!sync.barrier(c, &sh.abort, &sh.bar_phase)) {
                goto done;
            }
        }

        // ---- sequential parameter moves l = 1..N_p (Sec. 4.1) ----
        for (int l = 0; l < NP; ++l) {
            if (!((sh.free_mask >> l) & 1u)) continue;
            if (tid == 0) sh.par_prop[l] += 1ull;
            if (!sh.inbox[l]) continue;  // out of the prior box: rejected without compute
            if (tid == 0 && sync.lead()) chk_move(c);
            R pq[kMaxP];
#pragma unroll
            for (int q = 0; q < kMaxP; ++q) pq[q] = pr[q];
            apply_move<R, NT>(pq, sh, l);
            const R* Fc = (const R*)c.F[sh.fidx];
            R* Fn = (R*)c.F[sh.fidx ^ 1u];
            Fix3 part;
            fix_zero(part);
            const int64_t nend = min(n1, M);
            if (c.scheme == kSchemeRK4) {
                if constexpr (std::is_same<Model, HH<float>>::value)
                    param_terms_paired<NT>(c, kc, n0, nend, pq, beta, Fc, Fn, part);
                else
                    for (int64_t n = n0 + tid; n < nend; n += NT)
                        if (chk_site(c, 2, n)) fix_add(part, param_term<Model, R>(c, kc, n, pq, beta, Fc, Fn));
            } else {
                // trapezoid: F(x_n, p') of the tile (and of the next tile's
                // first site, recomputed here), then the residual changes
                R g[D];
                for (int64_t n = n0 + tid; n < n1; n += NT)
                    if (chk_site(c, 2, n)) trap_field<Model, R>(c, kc, n, pq, Fn, g);
                if (n1 <= M && tid == NT - 1) {
                    trap_field<Model, R>(c, kc, n1, pq, nullptr, g);
#pragma unroll
                    for (int a = 0; a < D; ++a) sh.halo[a] = g[a];
                }
                __syncthreads();
                for (int64_t n = n0 + tid; n < nend; n += NT) {
                    R gn1p[D];
#pragma unroll
                    for (int a = 0; a < D; ++a) gn1p[a] = (n + 1 < n1) ? Fn[a * c.ldf + n + 1] : sh.halo[a];
                    fix_add(part, trap_term<Model, R>(c, kc, n, beta, Fc, Fn, gn1p));
                }
            }
            // exact sum: CTA, then grid (accumulator slot), then the decision
            const unsigned slot = sh.nred % 3u;
            const Fix3 cta = fix_cta_sum<NT>(part, sh.wfix);
            if (tid == 0) sync.publish(c, slot, cta, &sh.cta_fix);
            if (!sync.barrier(c, &sh.abort, &sh.bar_phase)) goto done;
            if (tid == 0) {
                decide<R, NT>(sh, l, sync.total(c, slot, &sh.cta_fix));
                sync.recycle(c, slot);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kMaxP; ++q) pr[q] = sh.q_cur[q];
        }
        __syncthreads();

        {
            // ---- path statistics (Sec. 4.1): after N_init, every N_skip sweeps ----
            // (the residual of the tile's last site reads the next tile's first
            // site: a barrier keeps it unchanged until every CTA has recorded)
            const bool record = (s >= c.n_init) && ((s - c.n_init) % c.n_skip == 0);
            if (record) {
                record_sample<Model, R>(c, n0, n1, sync.lead(), sh.p, sh.J == 0, tid, NT, (const R*)c.F[sh.fidx]);
                if (!sync.barrier(c, &sh.abort, &sh.bar_phase)) goto done;
            }

            // ---- step-size adaptation during burn-in (Sec. 4.2) ----
            if (s < c.n_init && ((s + 1) % c.n_skip == 0)) {
                for (int64_t n = n0 + tid; n < n1; n += NT) {
                    const double fac = 1.0 + c.alpha * ((double)c.acc_win[n] / (double)c.n_skip - c.f_acc);
#pragma unroll
                    for (int a = 0; a < D; ++a) sig[a * c.ldx + n] = R((double)sig[a * c.ldx + n] * fac);
                    c.acc_win[n] = 0u;
                }
                if (tid == 0) adapt_params<NP>(c, sh);
            }
            end_sweep<NP>(c, sh, s, record, sync);
            if (Sync::tiled && sync.site_flags && tid == 0) flag_post(c, 1, ep);  // this tile is final for the sweep
        }
    }

done:
    store_chain_state(c, sh, sync, my_acc, my_prop, my_nf);
}

// ---- resident form ------------------------------------------------------------

// Values of site n for one parameter vector q: RK4, f(x_n) (n < M);
// trapezoid, F(x_n) and the neighbour's F(x_{n+1}) (n < M).
template <class Model, class R>
__device__ __forceinline__ void move_values(const Ctx& c, const Coef<R>& k, bool trap, bool has_next, const R* x,
                                            const R* xn, R drive, R drive1, const R* q, R* f, R* fn)
{
    if (!trap) {
        if (has_next) rk4_map<Model, R>(x, q, drive, k.dt, f);
    } else {
        Model::rhs(x, q, drive, f);
        if (has_next) Model::rhs(xn, q, drive1, fn);
    }
}

// Change of the model-error term eps_{n+1} when the cached values of n (and
// n+1 under the trapezoid rule) become f (fn).
template <class R, int D>
__device__ __forceinline__ R move_term(const Ctx& c, const Coef<R>& k, bool trap, const R* x, const R* xn,
                                       const R* g, const R* gn, const R* f, const R* fn, R beta)
{
    if constexpr (std::is_same<R, float>::value) {
        if (!trap) return rk4_term_lanes<float, D>(beta, k.Rf, xn, f, g);
    }
    R t = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (!trap) {
            t += beta * sqdiff<R>(k.Rf[a], xn[a] - f[a], xn[a] - g[a]);
        } else {
            const R e = eps_of<R>(c, k, x[a], xn[a], g[a], gn[a]);
            const R ep = eps_of<R>(c, k, x[a], xn[a], f[a], fn[a]);
            t += beta * sqdiff<R>(k.Rf[a], ep, e);
        }
    }
    return t;
}

// kTrap: the scheme (c.scheme) as a compile-time constant, so each launched
// kernel carries only its own scheme's branches of the parameter moves.
template <class Model, class R, int NT, bool kTrap, class Sync>
__device__ void sweep_chain_resident(const Ctx& c, int64_t n0, int64_t n1, int64_t n_sweeps, SweepShared<R, NT>& sh,
                                     const Sync& sync)
{
    constexpr int D = Model::D, NP = Model::NP;
    const int tid = threadIdx.x, lane = tid & 31;
    const Coef<R> kc(c);
    const int64_t M = c.M, T = n1 - n0;
    const int i = tid - 32;
    const int64_t n = n0 + i;
    const bool own = tid >= 32 && i < T;
    constexpr bool trap = kTrap;
    const int64_t clen = cache_len(c);
    const bool cached = own && n < clen;
    const bool has_next = own && n < M;          // site n carries eps_{n+1}
    const bool left_halo = own && i == 0 && n0 >= 1;
    const bool right_halo = own && i == T - 1 && n1 <= M;
    const int b = (int)blockIdx.x;
    R* X = (R*)c.X;
    R* sig = (R*)c.sig;

    // registers of the owned site
    R xr[D], sgr[D], gr[D], xh[D], gh[D];
    R yv = R(0), drive = R(0), drive1 = R(0);
    unsigned accw = 0u;
    unsigned long long my_acc[2] = {0ull, 0ull}, my_prop[2] = {0ull, 0ull}, my_nf = 0ull;
#pragma unroll
    for (int a = 0; a < D; ++a) xr[a] = sgr[a] = gr[a] = xh[a] = gh[a] = R(0);
    if (own) {
        const R* Fc = (const R*)c.F[sh.fidx];
        const R* I = (const R*)c.I;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            xr[a] = X[a * c.ldx + n];
            sgr[a] = sig[a * c.ldx + n];
            gr[a] = cached ? Fc[a * c.ldf + n] : R(0);
            sh.xs[a][i] = xr[a];
            sh.gs[a][i] = gr[a];
        }
        if (n >= 1) yv = ((const R*)c.y)[n];
        if (cached) drive = I[drive_index(c, n)];
        if (has_next && trap) drive1 = I[drive_index(c, n + 1)];
        accw = c.acc_win[n];
    }
    __syncthreads();

    bool odd_flag_wait = false;  // the previous sweep had no parameter barrier
    // this site's draws of the next sweep, formed during the last parameter
    // barrier of a sweep (they depend only on the counters)
    R zn[D], En = R(0);
#pragma unroll
    for (int a = 0; a < D; ++a) zn[a] = R(0);
    bool have_draws = false;
    for (int64_t k = 0; k < n_sweeps; ++k) {
        const long long s = sh.sweep;
        const unsigned long long ep = sh.ep0 + (unsigned long long)k + 1ull;
        // this sweep's parameter draws, evaluated before the launch by
        // param_draws_kernel (FP64 transcendental functions issue slowly on one
        // warp and would hold up the even phase)
        if (tid < NP && ((sh.free_mask >> tid) & 1u))
            set_param_proposal<Model, R, NT>(sh, tid, __ldg(c.pdraw + 2 * (k * NP + tid)),
                                             __ldg(c.pdraw + 2 * (k * NP + tid) + 1));
        const R beta = R(sh.beta);
        R pr[kMaxP];
#pragma unroll
        for (int q = 0; q < kMaxP; ++q) pr[q] = sh.q_cur[q];

        // ---- site phases: even sites, then odd sites (Sec. 4.1) ----
#pragma unroll
        for (int parity = 0; parity < 2; ++parity) {
            if (own && (int)(n & 1) == parity && chk_site(c, parity, n)) {
                // the proposal first: it needs no neighbour, so it overlaps the
                // halo wait of the tile's boundary sites
                R xp[D], gp[D], z[D], E;
                if (have_draws) {
#pragma unroll
                    for (int a = 0; a < D; ++a) z[a] = zn[a];
                    E = En;
                } else {
                    site_draw<Model, R>(c, s, n, z, E);
                }
                site_propose_from<Model, R>(c, kc, n, pr, xr, sgr, drive, z, xp, gp);
                Nbhd<R, D> nb;
                R xl[D], gl[D];
#pragma unroll
                for (int a = 0; a < D; ++a) xl[a] = gl[a] = R(0);
                const R* Fc = (const R*)c.F[sh.fidx];
                bool ok = true;
                if (left_halo) {
                    // the previous tile's last site: final after the last
                    // parameter barrier, or after its odd flag
                    if (odd_flag_wait && Sync::tiled) ok = flag_wait(c, 1, b - 1, ep - 1ull);
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        gl[a] = __ldcg(Fc + a * c.ldf + n0 - 1);
                        xl[a] = trap ? __ldcg(X + a * c.ldx + n0 - 1) : R(0);
                    }
                }
                if (right_halo) {
                    // the next tile's first site (even): final after its even phase
                    if (Sync::tiled) ok = flag_wait(c, 0, b + 1, ep);
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        xh[a] = __ldcg(X + a * c.ldx + n1);
                        gh[a] = trap ? __ldcg(Fc + a * c.ldf + n1) : R(0);
                    }
                }
                if (!ok) sh.abort = 1;
                if (n >= 1) {
                    nb.yn = yv;
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        nb.gprev[a] = (i > 0) ? sh.gs[a][i - 1] : gl[a];
                        nb.xprev[a] = trap ? ((i > 0) ? sh.xs[a][i - 1] : xl[a]) : R(0);
                    }
                }
#pragma unroll
                for (int a = 0; a < D; ++a) nb.gcur[a] = gr[a];
                if (n < M) {
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        nb.xn1[a] = (i + 1 < T) ? sh.xs[a][i + 1] : xh[a];
                        nb.gn1[a] = trap ? ((i + 1 < T) ? sh.gs[a][i + 1] : gh[a]) : R(0);
                    }
                }
                if (ok && site_decide<Model, R>(c, kc, n, xr, xp, gp, beta, E, nb, my_nf)) {
                    R* Fw = (R*)c.F[sh.fidx];
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        xr[a] = xp[a];
                        X[a * c.ldx + n] = xp[a];
                        sh.xs[a][i] = xp[a];
                    }
                    if (cached) {
#pragma unroll
                        for (int a = 0; a < D; ++a) {
                            gr[a] = gp[a];
                            Fw[a * c.ldf + n] = gp[a];
                            sh.gs[a][i] = gp[a];
                        }
                    }
                    accw += 1u;
                    my_acc[parity] += 1ull;
                }
                my_prop[parity] += 1ull;
            }
            __syncthreads();
            if (sh.abort) goto done;
            if (Sync::tiled && tid == 0 && parity == 0) flag_post(c, 0, ep);
        }

        have_draws = false;  // this sweep's draws are used
        {
            // ---- sequential parameter moves l = 1..N_p (Sec. 4.1) ----
            unsigned todo = 0u;
            for (int l = 0; l < NP; ++l) {
                if (!((sh.free_mask >> l) & 1u)) continue;
                if (sh.inbox[l]) todo |= 1u << l;
            }
            if (tid == 0)
                for (int l = 0; l < NP; ++l)
                    if ((sh.free_mask >> l) & 1u) sh.par_prop[l] += 1ull;
            // with no parameter barrier this sweep, the neighbours order on
            // the odd flag posted at its end
            odd_flag_wait = (todo == 0u);
            if (!odd_flag_wait) {
                // operands of the parameter phase: x_{n+1}, g_{n+1}
                R xn[D], gn[D], f[D], fn[D];
#pragma unroll
                for (int a = 0; a < D; ++a) xn[a] = gn[a] = f[a] = fn[a] = R(0);
                if (own) {
#pragma unroll
                    for (int a = 0; a < D; ++a) {
                        xn[a] = (i + 1 < T) ? sh.xs[a][i + 1] : xh[a];
                        gn[a] = (i + 1 < T) ? sh.gs[a][i + 1] : gh[a];
                    }
                }
                // first move: no decision pending
                int l = __ffs(todo) - 1;
                Fix3 mine;
                fix_zero(mine);
                if (own) {
                    R q[kMaxP];
#pragma unroll
                    for (int j = 0; j < kMaxP; ++j) q[j] = pr[j];
                    apply_move<R, NT>(q, sh, l);
                    move_values<Model, R>(c, kc, trap, has_next, xr, xn, drive, drive1, q, f, fn);
                    if (has_next) fix_add(mine, move_term<R, D>(c, kc, trap, xr, xn, gr, gn, f, fn, beta));
                    if (cached && chk_site(c, 2, n)) {
                        R* Fn = (R*)c.F[sh.fidx ^ 1u];
#pragma unroll
                        for (int a = 0; a < D; ++a) Fn[a * c.ldf + n] = f[a];
                    }
                }
                // from the second move on, the CTA sums of the move's terms for
                // both outcomes of the decision before were formed during that
                // decision's barrier (buffer spec_buf)
                bool spec_sums = false;
                int spec_buf = 0;
                while (true) {
                    todo &= todo - 1u;
                    const int l2 = todo ? __ffs(todo) - 1 : -1;
                    R fA[D], fnA[D], fR[D], fnR[D];
                    Fix3 tA, tR;  // move l2's term of this site for each outcome of move l
                    fix_zero(tA);
                    fix_zero(tR);
                    const unsigned slot = sh.nred % 3u;
                    Fix3 cta;
                    if (spec_sums) {
                        // before the sweep's last barrier, the site threads'
                        // cache stores of this move (after the decision
                        // before) are ordered ahead of the arrival: the next
                        // sweep's halo reads of other CTAs rely on that barrier
                        if (l2 < 0) __syncthreads();
                        fix_zero(cta);
                        if (tid == 0) cta = sh.cta_spec[spec_buf][sh.last_acc ? 0 : 1];
                        spec_buf ^= 1;
                    } else {
                        cta = fix_cta_sum<NT>(mine, sh.wfix);  // exact CTA sum (a CTA barrier inside)
                    }
                    if (tid < 32) {
                        // thread 0: publish, grid barrier, total, decide
                        if (lane == 0) {
                            sync.publish(c, slot, cta, &sh.cta_fix);
                            if (!sync.arrive_wait(c, &sh.bar_phase)) sh.abort = 1;
                            else {
                                decide<R, NT>(sh, l, sync.total(c, slot, &sh.cta_fix));
                                sync.recycle(c, slot);
                                if (sync.lead()) chk_move(c);
                            }
                        }
                    } else if (l2 >= 0) {
                        if (own) {
                            // speculation: move l2's values for both outcomes of
                            // move l.  FP32 HH under the RK4 scheme: both maps as
                            // the two lanes of one packed evaluation (lane x:
                            // reject, lane y: accept), each lane bit for bit the
                            // single map.  Otherwise one map instance evaluated
                            // twice (two inlined copies would share
                            // subexpressions, and the compiler would fuse
                            // multiply-adds differently from the general form's
                            // single map).
                            bool spec_done = false;
                            if constexpr (std::is_same<Model, HH<float>>::value) {
                                if (!trap) {
                                    spec_done = true;
                                    if (has_next) {
                                        R qR[kMaxP], qA[kMaxP];
#pragma unroll
                                        for (int j = 0; j < kMaxP; ++j) qR[j] = pr[j];
                                        apply_move<R, NT>(qR, sh, l2);
#pragma unroll
                                        for (int j = 0; j < kMaxP; ++j) qA[j] = qR[j];
                                        apply_move<R, NT>(qA, sh, l);
                                        float2 q2[kMaxP], x2[D], f2[D];
#pragma unroll
                                        for (int j = 0; j < kMaxP; ++j) q2[j] = make_float2(qR[j], qA[j]);
#pragma unroll
                                        for (int a = 0; a < D; ++a) x2[a] = splat<float2>(xr[a]);
                                        hh_rk4_lanes<float2>(x2, q2, splat<float2>(drive), splat<float2>(kc.dt),
                                                             splat<float2>(__fmul_rn(0.5f, kc.dt)),
                                                             splat<float2>(__fdiv_rn(kc.dt, 6.0f)), f2);
#pragma unroll
                                        for (int a = 0; a < D; ++a) {
                                            fR[a] = f2[a].x;
                                            fA[a] = f2[a].y;
                                        }
                                    }
#pragma unroll
                                    for (int a = 0; a < D; ++a) fnA[a] = fnR[a] = R(0);
                                }
                            }
#pragma unroll 1
                            for (int o = 0; o < (spec_done ? 0 : 2); ++o) {
                                R q[kMaxP], f2[D], fn2[D];
#pragma unroll
                                for (int j = 0; j < kMaxP; ++j) q[j] = pr[j];
                                apply_move<R, NT>(q, sh, l2);
                                if (o == 1) apply_move<R, NT>(q, sh, l);
                                move_values<Model, R>(c, kc, trap, has_next, xr, xn, drive, drive1, q, f2, fn2);
#pragma unroll
                                for (int a = 0; a < D; ++a) {
                                    if (o == 1) {
                                        fA[a] = f2[a];
                                        fnA[a] = fn2[a];
                                    } else {
                                        fR[a] = f2[a];
                                        fnR[a] = fn2[a];
                                    }
                                }
                            }
                            // and move l2's term for each outcome: accepting l
                            // makes move l's values (f, fn) this site's cache
                            if (has_next) {
                                fix_add(tA, move_term<R, D>(c, kc, trap, xr, xn, f, fn, fA, fnA, beta));
                                fix_add(tR, move_term<R, D>(c, kc, trap, xr, xn, gr, gn, fR, fnR, beta));
                            }
                        }
                        // CTA sums of those terms for both outcomes, by the site
                        // warps alone (named barrier 1; warp 0 holds no site
                        // and is in the grid barrier) -- exact, so the same
                        // total as the sum after the decision
                        const Fix3 wA = fix_warp_sum(tA), wR = fix_warp_sum(tR);
                        if (lane == 0) {
                            sh.wspec[0][tid >> 5] = wA;
                            sh.wspec[1][tid >> 5] = wR;
                        }
                        asm volatile("bar.sync 1, %0;" ::"r"(NT - 32) : "memory");
                        if (tid < 64) {
                            Fix3 a, r;
                            fix_zero(a);
                            fix_zero(r);
                            if (lane < NT / 32 - 1) {
                                a = sh.wspec[0][lane + 1];
                                r = sh.wspec[1][lane + 1];
                            }
                            a = fix_warp_sum(a);
                            r = fix_warp_sum(r);
                            fix_normalize(a);
                            fix_normalize(r);
                            if (lane == 0) {
                                sh.cta_spec[spec_buf][0] = a;
                                sh.cta_spec[spec_buf][1] = r;
                            }
                        }
                    } else if (own) {
                        // the sweep's last move: the site threads have no
                        // speculation to do during its barrier, so they draw
                        // this site's move of the next sweep
                        site_draw<Model, R>(c, s + 1, n, zn, En);
                        have_draws = true;
                    }
                    __syncthreads();
                    if (sh.abort) goto done;
                    const bool acc = sh.last_acc != 0;
#pragma unroll
                    for (int j = 0; j < kMaxP; ++j) pr[j] = sh.q_cur[j];
                    if (acc) {
#pragma unroll
                        for (int a = 0; a < D; ++a) {
                            gr[a] = f[a];
                            gn[a] = fn[a];
                        }
                    }
                    if (l2 < 0) break;
                    l = l2;
                    spec_sums = true;
                    if (own) {
#pragma unroll
                        for (int a = 0; a < D; ++a) {
                            f[a] = acc ? fA[a] : fR[a];
                            fn[a] = acc ? fnA[a] : fnR[a];
                        }
                        if (cached && chk_site(c, 2, n)) {
                            R* Fn = (R*)c.F[sh.fidx ^ 1u];
#pragma unroll
                            for (int a = 0; a < D; ++a) Fn[a * c.ldf + n] = f[a];
                        }
                    }
                }
                if (own) {
#pragma unroll
                    for (int a = 0; a < D; ++a) sh.gs[a][i] = gr[a];
                }
            }
        }
        __syncthreads();

        {
            // ---- path statistics (Sec. 4.1): after N_init, every N_skip sweeps ----
            // (the residual of the tile's last site reads the next tile's first
            // site: a barrier keeps it unchanged until every CTA has recorded)
            const bool record = (s >= c.n_init) && ((s - c.n_init) % c.n_skip == 0);
            if (record) {
                record_sample<Model, R>(c, n0, n1, sync.lead(), sh.p, sh.J == 0, tid, NT, (const R*)c.F[sh.fidx]);
                if (!sync.barrier(c, &sh.abort, &sh.bar_phase)) goto done;
            }

            // ---- step-size adaptation during burn-in (Sec. 4.2) ----
            if (s < c.n_init && ((s + 1) % c.n_skip == 0)) {
                if (own) {
                    const double fac = 1.0 + c.alpha * ((double)accw / (double)c.n_skip - c.f_acc);
#pragma unroll
                    for (int a = 0; a < D; ++a) sgr[a] = R((double)sgr[a] * fac);
                    accw = 0u;
                }
                if (tid == 0) adapt_params<NP>(c, sh);
            }
            end_sweep<NP>(c, sh, s, record, sync);
            if (Sync::tiled && odd_flag_wait && tid == 0) flag_post(c, 1, ep);
        }
    }

done:
    if (own) {
#pragma unroll
        for (int a = 0; a < D; ++a) sig[a * c.ldx + n] = sgr[a];
        c.acc_win[n] = accw;
    }
    store_chain_state(c, sh, sync, my_acc, my_prop, my_nf);
}

template <class Model, class R, int NT, class Sync>
__device__ void sweep_chain(const Ctx& c, int64_t n0, int64_t n1, int64_t n_sweeps, SweepShared<R, NT>& sh,
                            const Sync& sync)
{
    if (threadIdx.x == 0) load_chain_state<Model, R, NT>(c, sh);
    __syncthreads();
    sweep_chain_general<Model, R, NT>(c, n0, n1, n_sweeps, sh, sync);
}

// FP32: two resident CTAs an SM (at most 128 registers a thread).
template <class R> struct SweepBounds { static constexpr int min_blocks = 1; };
template <> struct SweepBounds<float> { static constexpr int min_blocks = 2; };

template <class Model, class R>
__global__ void __launch_bounds__(kSweepBlock, SweepBounds<R>::min_blocks) sweep_kernel(Ctx c, int64_t n_sweeps)
{
    __shared__ SweepShared<R, kSweepBlock> sh;
    const int64_t n0 = (int64_t)blockIdx.x * c.tile;
    const int64_t n1 = min(n0 + c.tile, c.M + 1);
    sweep_chain<Model, R, kSweepBlock>(c, n0, n1, n_sweeps, sh, GridSync{(int)blockIdx.x, (int)gridDim.x, 1});
}

// The parameter draws of the next n sweeps of a chain: out[2 (k NP + l)] = z,
// out[2 (k NP + l) + 1] = -log u for sweep st->sweep + k -- the same values
// the sweep draws itself (param_draw).  Four lanes a (sweep, parameter) take
// the three independent FP64 chains in parallel (FP64 issues slowly on this
// part, so the draws' latency, ahead of every resident launch, is the longest
// chain): the Box-Muller radius sqrt(-2 log u1), the cosine cos(2 pi u2) and
// -log u of the accept uniform; z = radius * cosine as in the one-thread form.
// Also zeroes the three rotating accumulator slots of the exact sums.
template <int NP>
__global__ void __launch_bounds__(256) param_draws_kernel(Ctx c, int64_t n, double* out)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 12) ((unsigned long long*)c.partials)[t] = 0ull;
    const int64_t idx = t >> 2;  // (sweep, parameter)
    const int role = (int)(t & 3);
    const bool valid = idx < n * NP;
    const int l = (int)(idx % NP);
    const long long s = c.st->sweep + idx / NP;
    const bool draw = valid && ((c.st->free_mask >> l) & 1u);
    double v = 0.0;
    if (draw) {
        if (role < 2) {
            const uint4 wz = draw_block(c.seed, c.chain, (uint64_t)s, (uint32_t)l, kKindParam, 0u);
            if (c.proposal == kProposalUniform) {
                v = role == 0 ? 2.0 * u01d(wz.x, wz.y) - 1.0 : 1.0;
            } else if (role == 0) {
                v = sqrt(-2.0 * log(u01d(wz.x, wz.y)));
            } else {
                double sn, cs;
                sincospi(2.0 * u01d(wz.z, wz.w), &sn, &cs);
                v = cs;
            }
        } else if (role == 2) {
            const uint4 w = draw_block(c.seed, c.chain, (uint64_t)s, (uint32_t)l, kKindParam, 1u);
            v = -log(u01d(w.x, w.y));
        }
    }
    // lanes 4j..4j+3 of a warp hold one (sweep, parameter)
    const double cosv = __shfl_down_sync(0xffffffffu, v, 1);
    const double elog = __shfl_down_sync(0xffffffffu, v, 2);
    if (valid && role == 0) {
        out[2 * idx] = draw ? (c.proposal == kProposalUniform ? v : v * cosv) : 0.0;
        out[2 * idx + 1] = draw ? elog : 0.0;
    }
}

// Resident form (FP32-mixed): tiles of at most kSweepBlock - 32 sites, even
// when there are several.  It evaluates two maps per site and parameter move
// to take them off the critical path, which pays where the sweep is bound by
// synchronisation latency (FP32 arithmetic at moderate M), not by arithmetic
// throughput (FP64).
template <class Model, bool kTrap>
__global__ void __launch_bounds__(kSweepBlock, 1) sweep_resident_kernel(Ctx c, int64_t n_sweeps)
{
    __shared__ SweepShared<float, kSweepBlock> sh;
    const int64_t n0 = (int64_t)blockIdx.x * c.tile;
    const int64_t n1 = min(n0 + c.tile, c.M + 1);
    if (threadIdx.x == 0) load_chain_state<Model, float, kSweepBlock>(c, sh);
    __syncthreads();
    sweep_chain_resident<Model, float, kSweepBlock, kTrap>(c, n0, n1, n_sweeps, sh,
                                                           GridSync{(int)blockIdx.x, (int)gridDim.x});
}

bool resident_fits(int prec, int64_t tile, int grid)
{
    return prec == 1 && tile <= kSweepBlock - 32 && (grid == 1 || (tile & 1) == 0);
}

// Many chains in one launch: CTA b runs, one after another, the items
// items[first[b] .. first[b+1]): a whole chain (CTA-local synchronisation), or
// one tile of a long chain split over `size` CTAs, which then synchronise on
// the chain's own barrier word and exact-sum slots (bounded waits).  Every
// CTA's items follow one global order, so the CTAs of a split chain meet
// without a cycle of waits; the launch is cooperative whenever a chain is
// split.  Counters are keyed by the chain, never the CTA, so a chain's bits do
// not depend on how it is tiled.
// FP32: at least 512 / NT resident CTAs per SM (at most 128 registers a thread).
template <class R, int NT> struct BatchBounds { static constexpr int min_blocks = 1; };
template <int NT> struct BatchBounds<float, NT> { static constexpr int min_blocks = 512 / NT; };

// kSplit = false: a launch whose items are all whole chains (compiled without
// the split path, which would otherwise share its register budget).
template <class Model, class R, int NT, bool kSplit>
__global__ void __launch_bounds__(NT, BatchBounds<R, NT>::min_blocks)
    batch_sweep_kernel(const Ctx* chains, const int* first, const BatchItem* items, int64_t n_sweeps, uint64_t seed)
{
    __shared__ SweepShared<R, NT> sh;
    __shared__ Ctx cs;  // the current chain's context, read from shared memory
    for (int i = first[blockIdx.x]; i < first[blockIdx.x + 1]; ++i) {
        const BatchItem it = items[i];
        if (threadIdx.x == 0) {
            cs = chains[it.chain];
            cs.seed = seed;
        }
        __syncthreads();
        if (it.size <= 1) {
            sweep_chain<Model, R, NT>(cs, 0, cs.M + 1, n_sweeps, sh, BlockSync{});
        } else if constexpr (!kSplit) {
            // a split item in a launch planned without splits: refused (the
            // host never plans one)
            if (threadIdx.x == 0) atomicOr(&cs.st->status, kStatusBounds);
        } else {
            // tile `rank` of `size` tiles of even length (as a chain's own launch tiles it)
            int64_t tile = (cs.M + 1 + it.size - 1) / it.size;
            tile += tile & 1;
            const int64_t n0 = min((int64_t)it.rank * tile, cs.M + 1), n1 = min(n0 + tile, cs.M + 1);
            const GridSync sync{it.rank, it.size};
            if (threadIdx.x == 0) {
                load_chain_state<Model, R, NT>(cs, sh);
                // the exact-sum slots start at zero: rank 0 clears them before
                // the group's first barrier
                if (it.rank == 0)
                    for (int j = 0; j < 12; ++j) __stcg((unsigned long long*)cs.partials + j, 0ull);
            }
            __syncthreads();
            if (sync.barrier(cs, &sh.abort, &sh.bar_phase))
                sweep_chain_general<Model, R, NT>(cs, n0, n1, n_sweeps, sh, sync);
        }
        __syncthreads();
    }
}

template <class Model, class R> struct SweepKernels {
    static const void* general() { return (const void*)sweep_kernel<Model, R>; }
    static const void* resident(int) { return nullptr; }
};
template <class Model> struct SweepKernels<Model, float> {
    static const void* general() { return (const void*)sweep_kernel<Model, float>; }
    static const void* resident(int scheme)
    {
        return scheme == kSchemeRK4 ? (const void*)sweep_resident_kernel<Model, false>
                                    : (const void*)sweep_resident_kernel<Model, true>;
    }
};

// Opt a kernel in to `bytes` of dynamic shared memory (above the default
// limit once the static part is added); once per kernel, remembered by the
// kernel's address (kernels of one signature are distinct entries), under a
// lock: handles may be driven from several host threads.
static cudaError_t allow_dynamic_smem(const void* kernel, int bytes)
{
    if (bytes == 0) return cudaSuccess;
    static std::mutex mu;
    static std::vector<std::pair<const void*, int>> done;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto& d : done)
        if (d.first == kernel && d.second >= bytes) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.emplace_back(kernel, bytes);
    return e;
}

template <class Model, class R>
static cudaError_t launch_sweep_t(const Ctx& c, int64_t n_sweeps, int grid, int resident, cudaStream_t s)
{
    Ctx cc = c;
    int64_t ns = n_sweeps;
    void* args[] = {(void*)&cc, (void*)&ns};
    const bool res = resident && resident_fits(prec_of<R>(), c.tile, grid) && c.pdraw && n_sweeps <= kDrawChunk;
    if (res && n_sweeps > 0) {
        // the draws kernel also zeroes the accumulator slots of the exact sums
        const int64_t nt = 4 * n_sweeps * Model::NP;
        param_draws_kernel<Model::NP><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(c, n_sweeps, const_cast<double*>(c.pdraw));
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    } else {
        // the three accumulator slots of the exact parameter-move sums start at zero
        const cudaError_t e = cudaMemsetAsync(c.partials, 0, 12 * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    const void* k = res ? SweepKernels<Model, R>::resident(c.scheme) : SweepKernels<Model, R>::general();
    const int smem = res ? 0 : StageBytes<Model, R, kSweepBlock>::value;
    const cudaError_t e = allow_dynamic_smem((const void*)sweep_kernel<Model, R>, StageBytes<Model, R, kSweepBlock>::value);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kSweepBlock), args, (size_t)smem, s);
}

static int max_grid_of(const void* k, int device, int smem)
{
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kSweepBlock, (size_t)smem) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return per_sm * sms;
}

template <class Model, class R>
static int max_grid_t(int device, int resident)
{
    if (allow_dynamic_smem((const void*)sweep_kernel<Model, R>, StageBytes<Model, R, kSweepBlock>::value) != cudaSuccess) return 0;
    if (resident) {
        // the smaller capacity of the two scheme variants
        const void* k0 = SweepKernels<Model, R>::resident(kSchemeRK4);
        const void* k1 = SweepKernels<Model, R>::resident(kSchemeTrapezoid);
        return (k0 && k1) ? std::min(max_grid_of(k0, device, 0), max_grid_of(k1, device, 0)) : 0;
    }
    return max_grid_of(SweepKernels<Model, R>::general(), device, StageBytes<Model, R, kSweepBlock>::value);
}

cudaError_t launch_sweep(int model, int prec, const Ctx& c, int64_t n_sweeps, int grid, int resident, cudaStream_t s)
{
    PIMC_DISPATCH(launch_sweep_t, c, n_sweeps, grid, resident, s);
}

int sweep_max_grid(int model, int prec, int device, int resident)
{
    PIMC_DISPATCH(max_grid_t, device, resident);
}

// ---- batched launch --------------------------------------------------------

template <class Model, class R, int NT>
static cudaError_t batch_t(const Ctx* chains, const int* first, const BatchItem* items, int n_ctas, int64_t n_sweeps,
                           uint64_t seed, bool cooperative, cudaStream_t s)
{
    constexpr int smem = StageBytes<Model, R, NT>::value;
    if (!cooperative) {
        // no split chain: the kernel without the split path
        const cudaError_t e = allow_dynamic_smem((const void*)batch_sweep_kernel<Model, R, NT, false>, smem);
        if (e != cudaSuccess) return e;
        batch_sweep_kernel<Model, R, NT, false><<<n_ctas, NT, smem, s>>>(chains, first, items, n_sweeps, seed);
        return cudaGetLastError();
    }
    const cudaError_t e = allow_dynamic_smem((const void*)batch_sweep_kernel<Model, R, NT, true>, smem);
    if (e != cudaSuccess) return e;
    int64_t ns = n_sweeps;
    uint64_t sd = seed;
    void* args[] = {(void*)&chains, (void*)&first, (void*)&items, (void*)&ns, (void*)&sd};
    return cudaLaunchCooperativeKernel((const void*)batch_sweep_kernel<Model, R, NT, true>, dim3(n_ctas), dim3(NT), args,
                                       (size_t)smem, s);
}

template <class Model, class R, int NT> static int batch_occ_t()
{
    constexpr int smem = StageBytes<Model, R, NT>::value;
    if (allow_dynamic_smem((const void*)batch_sweep_kernel<Model, R, NT, true>, smem) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_sweep_kernel<Model, R, NT, true>, NT, (size_t)smem) !=
        cudaSuccess)
        return 0;
    return per_sm;
}

#define PIMC_BATCH_DISPATCH(FN, ...)                                                               \
    do {                                                                                           \
        if (nt == 128) {                                                                           \
            if (prec == 0) {                                                                       \
                if (model == 0) return FN<HH<double>, double, 128>(__VA_ARGS__);                   \
                if (model == 1) return FN<LinGauss<double>, double, 128>(__VA_ARGS__);             \
                if (model == 3) return FN<HHPaper<double>, double, 128>(__VA_ARGS__);              \
                return FN<Toy1D<double>, double, 128>(__VA_ARGS__);                                \
            }                                                                                      \
            if (model == 0) return FN<HH<float>, float, 128>(__VA_ARGS__);                         \
            if (model == 1) return FN<LinGauss<float>, float, 128>(__VA_ARGS__);                   \
            if (model == 3) return FN<HHPaper<float>, float, 128>(__VA_ARGS__);                    \
            return FN<Toy1D<float>, float, 128>(__VA_ARGS__);                                      \
        }                                                                                          \
        if (prec == 0) {                                                                           \
            if (model == 0) return FN<HH<double>, double, 256>(__VA_ARGS__);                       \
            if (model == 1) return FN<LinGauss<double>, double, 256>(__VA_ARGS__);                 \
            if (model == 3) return FN<HHPaper<double>, double, 256>(__VA_ARGS__);                  \
            return FN<Toy1D<double>, double, 256>(__VA_ARGS__);                                    \
        }                                                                                          \
        if (model == 0) return FN<HH<float>, float, 256>(__VA_ARGS__);                             \
        if (model == 1) return FN<LinGauss<float>, float, 256>(__VA_ARGS__);                       \
        if (model == 3) return FN<HHPaper<float>, float, 256>(__VA_ARGS__);                        \
        return FN<Toy1D<float>, float, 256>(__VA_ARGS__);                                          \
    } while (0)

cudaError_t launch_batch_sweep(int model, int prec, int nt, const Ctx* chains, const int* first,
                               const BatchItem* items, int n_ctas, int64_t n_sweeps, uint64_t seed, bool cooperative,
                               cudaStream_t s)
{
    PIMC_BATCH_DISPATCH(batch_t, chains, first, items, n_ctas, n_sweeps, seed, cooperative, s);
}

int batch_ctas_per_sm(int model, int prec, int nt) { PIMC_BATCH_DISPATCH(batch_occ_t); }

// ---- diagnostic kernels sharing the sweep's per-site code ------------------

template <class Model, class R>
__global__ void __launch_bounds__(kBlock) site_delta_kernel(Ctx c, const double* Xp, double beta, double* dA)
{
    constexpr int D = Model::D;
    const int64_t n = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (n > c.M) return;
    const R* X = (const R*)c.X;
    const R* Fc = (const R*)c.F[c.st->fidx];
    const Coef<R> kc(c);
    R pr[kMaxP];
    Model::prep(c.st->p, pr);
    R x[D], xp[D], fp[D];
    Nbhd<R, D> nb;
    for (int a = 0; a < D; ++a) {
        x[a] = X[a * c.ldx + n];
        xp[a] = R(Xp[a * (c.M + 1) + n]);
    }
    load_nbhd<Model, R>(c, n, Fc, nb);
    for (int a = 0; a < D; ++a) fp[a] = R(0);
    if (n < cache_len(c)) cache_value<Model, R>(c, kc, xp, pr, n, fp);
    dA[n] = (double)site_delta<Model, R>(c, kc, n, x, xp, fp, R(beta), nb);
}

// Full-path parameter change of action, summed exactly like the sweep's
// parameter moves (Fix3): per-CTA sums added into an accumulator slot, then
// the last CTA to finish (ticket) rounds the total once.  For the trapezoid
// rule the new field of every site is written first (trap_field_kernel) and
// read by this kernel.
template <class Model, class R>
__global__ void __launch_bounds__(kBlock) param_delta_kernel(Ctx c, int l, double pl_new, double beta, double* out)
{
    __shared__ Fix3 wfix[kBlock / 32];
    __shared__ int last;
    const R* Fc = (const R*)c.F[c.st->fidx];
    R* Fn = (R*)c.F[c.st->fidx ^ 1u];
    double pd[kMaxP];
#pragma unroll
    for (int q = 0; q < kMaxP; ++q) pd[q] = (q == l) ? pl_new : c.st->p[q];
    R pq[kMaxP];
    Model::prep(pd, pq);
    const Coef<R> kc(c);
    Fix3 part;
    fix_zero(part);
    for (int64_t n = (int64_t)blockIdx.x * kBlock + threadIdx.x; n < c.M; n += (int64_t)gridDim.x * kBlock) {
        if (c.scheme == kSchemeRK4) {
            fix_add(part, param_term<Model, R>(c, kc, n, pq, R(beta), Fc, Fn));
        } else {
            R gn1p[Model::D];
            for (int a = 0; a < Model::D; ++a) gn1p[a] = Fn[a * c.ldf + n + 1];
            fix_add(part, trap_term<Model, R>(c, kc, n, R(beta), Fc, Fn, gn1p));
        }
    }
    const Fix3 cta = fix_cta_sum<kBlock>(part, wfix);
    unsigned long long* acc = (unsigned long long*)c.red;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j) atomicAdd(acc + j, (unsigned long long)cta.c[j]);
        if (cta.flags) atomicOr(acc + 3, cta.flags);
        __threadfence();
        last = (atomicAdd(c.ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        Fix3 t;
#pragma unroll
        for (int j = 0; j < 3; ++j) t.c[j] = (long long)__ldcg(acc + j);
        t.flags = __ldcg(acc + 3);
        *out = fix_value(t);
        *c.ticket = 0u;
    }
}

// The exact sum of n terms by one CTA (the test hook of the Fix3 arithmetic;
// acc128: FP32 terms through the per-thread 128-bit accumulator, as the
// general form's parameter moves add them).
template <class T, bool acc128>
__global__ void __launch_bounds__(256) fix_sum_kernel(const double* t, int64_t n, double* out)
{
    __shared__ Fix3 wfix[256 / 32];
    Fix3 f;
    fix_zero(f);
    if constexpr (acc128) {
        Acc128 a{0ull, 0ull};
        for (int64_t i = threadIdx.x; i < n; i += 256) acc_add(a, f, (float)t[i]);
        acc_fold(a, f);
    } else {
        for (int64_t i = threadIdx.x; i < n; i += 256) fix_add(f, (T)t[i]);
    }
    const Fix3 s = fix_cta_sum<256>(f, wfix);
    if (threadIdx.x == 0) *out = fix_value(s);
}

// The FP32 HH map (one RK4 step) of n sites in the single-lane form, written
// to out[4][n] as FP64, and of the pairs (2i, 2i + 1) in the packed f32x2
// form; *mismatch counts the pair components whose bits differ from the
// single-lane map (the test hook of the lane form).
__global__ void __launch_bounds__(256) lane_maps_kernel(const double* X, const double* I, const double* p, double dt,
                                                        int64_t n, double* out, unsigned* mismatch)
{
    const int64_t n0 = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (n0 >= n) return;
    const bool two = n0 + 1 < n;
    float q[kMaxP];
    HH<float>::prep(p, q);
    const float dtf = (float)dt;
    float x[2][4], f[2][4], drive[2];
#pragma unroll
    for (int L = 0; L < 2; ++L) {
        const int64_t nn = (L == 1 && two) ? n0 + 1 : n0;
#pragma unroll
        for (int a = 0; a < 4; ++a) x[L][a] = (float)X[a * n + nn];
        drive[L] = (float)I[nn];
        rk4_map<HH<float>, float>(x[L], q, drive[L], dtf, f[L]);
    }
    float2 x2[4], q2[kMaxP], f2[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) x2[a] = make_float2(x[0][a], x[1][a]);
#pragma unroll
    for (int j = 0; j < kMaxP; ++j) q2[j] = splat<float2>(q[j]);
    hh_rk4_lanes<float2>(x2, q2, make_float2(drive[0], drive[1]), splat<float2>(dtf),
                         splat<float2>(__fmul_rn(0.5f, dtf)), splat<float2>(__fdiv_rn(dtf, 6.0f)), f2);
    unsigned bad = 0u;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        bad += __float_as_uint(f2[a].x) != __float_as_uint(f[0][a]) ? 1u : 0u;
        bad += (two && __float_as_uint(f2[a].y) != __float_as_uint(f[1][a])) ? 1u : 0u;
        out[a * n + n0] = (double)f[0][a];
        if (two) out[a * n + n0 + 1] = (double)f[1][a];
    }
    if (bad) atomicAdd(mismatch, bad);
}

cudaError_t launch_lane_maps(const double* X, const double* I, const double* p, double dt, int64_t n, double* out,
                             unsigned* mismatch, cudaStream_t s)
{
    const int64_t pairs = (n + 1) / 2;
    lane_maps_kernel<<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(X, I, p, dt, n, out, mismatch);
    return cudaGetLastError();
}

cudaError_t launch_fix_sum(const double* t, int64_t n, int as_float, double* out, cudaStream_t s)
{
    if (as_float == 2) fix_sum_kernel<float, true><<<1, 256, 0, s>>>(t, n, out);
    else if (as_float) fix_sum_kernel<float, false><<<1, 256, 0, s>>>(t, n, out);
    else fix_sum_kernel<double, false><<<1, 256, 0, s>>>(t, n, out);
    return cudaGetLastError();
}

template <class Model, class R>
__global__ void trap_field_kernel(Ctx c, int l, double pl_new)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n > c.M) return;
    double pd[kMaxP];
    for (int q = 0; q < kMaxP; ++q) pd[q] = c.st->p[q];
    pd[l] = pl_new;
    R pq[kMaxP], g[Model::D];
    Model::prep(pd, pq);
    const Coef<R> kc(c);
    trap_field<Model, R>(c, kc, n, pq, (R*)c.F[c.st->fidx ^ 1u], g);
}

template <class Model, class R>
static cudaError_t site_delta_t(const Ctx& c, const double* Xp, double beta, double* dA, cudaStream_t s)
{
    const int grid = (int)((c.M + 1 + kBlock - 1) / kBlock);
    site_delta_kernel<Model, R><<<grid, kBlock, 0, s>>>(c, Xp, beta, dA);
    return cudaGetLastError();
}

template <class Model, class R>
static cudaError_t param_delta_t(const Ctx& c, int l, double pl, double beta, double* out, cudaStream_t s)
{
    if (c.scheme != kSchemeRK4) {
        trap_field_kernel<Model, R><<<(unsigned)((c.M + 1 + 255) / 256), 256, 0, s>>>(c, l, pl);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    int grid = (int)((c.M + kBlock - 1) / kBlock);
    if (grid > kMaxGrid) grid = kMaxGrid;
    if (grid < 1) grid = 1;
    const cudaError_t e = cudaMemsetAsync(c.red, 0, 4 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    param_delta_kernel<Model, R><<<grid, kBlock, 0, s>>>(c, l, pl, beta, out);
    return cudaGetLastError();
}

cudaError_t launch_site_delta(int model, int prec, const Ctx& c, const double* Xp, double beta, double* dA,
                              cudaStream_t s)
{
    PIMC_DISPATCH(site_delta_t, c, Xp, beta, dA, s);
}

cudaError_t launch_param_delta(int model, int prec, const Ctx& c, int l, double pl_new, double beta,
                               double* out, cudaStream_t s)
{
    PIMC_DISPATCH(param_delta_t, c, l, pl_new, beta, out, s);
}

}  // namespace pimc
