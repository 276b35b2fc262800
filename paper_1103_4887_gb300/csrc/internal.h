// Internal interface between the host runtime (runtime.cu) and the kernels
// (sweep.cu, ops.cu).  Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pimc {

constexpr int kBlock = 128;          // threads per CTA of the whole-path kernels
constexpr int kSweepBlock = 256;     // threads per CTA of the sweep kernel
constexpr int kMaxParams = 8;
constexpr int kMaxGrid = 4096;       // upper bound on CTAs of a launch (partials capacity)
constexpr int kMaxSel = 64;          // histogram components
constexpr int kMaxBins = 4096;
constexpr int kDrawChunk = 4096;   // sweeps a launch (the parameter-draw buffer's capacity)
constexpr int kRedStride = 16;     // per-CTA double slots of the single-pass reductions' scratch

// Scalar sampler state living in device memory.  The sweep kernel keeps a
// per-CTA copy in shared memory; every CTA evolves it identically (same draws,
// same fixed-order sums) and CTA 0 writes it back at the end of a launch.
struct DevState {
    double p[8], lo[8], hi[8], sigp[8];
    double beta;
    long long sweep, J;
    unsigned fidx, free_mask;
    unsigned accp_win[8];
    unsigned long long site_acc[2], site_prop[2], par_acc[8], par_prop[8], nonfinite;
    long long tr_n;  // parameter vectors written to the trace ring so far
    int status;   // sticky error bits (kStatusTimeout, kStatusBounds)
    int abort;    // set by a CTA whose bounded wait expired; all CTAs leave
};

constexpr int kStatusTimeout = 1;
constexpr int kStatusBounds = 2;  // checked builds: a site index outside [0, M] was met (access skipped)

// Everything a kernel needs, passed by value.
struct Ctx {
    int64_t M, ldx, ldf;          // sites 0..M; row strides of [D][ldx] and [D][ldf] arrays
    int scheme;                   // kSchemeRK4 or kSchemeTrapezoid
    int proposal;                 // kProposalGauss or kProposalUniform
    double dt, Rm, Rf[4];
    void* X;                      // R[D][ldx]
    void* F[2];                   // R[D][ldf]: cached f(x_n) or F(x_n), double-buffered (Sec. 4.3)
    const void* y;                // R[ldx]
    const void* I;                // R[ldf]
    void* sig;                    // R[D][ldx]
    uint32_t* acc_win;            // [ldx] accepted moves per site in the adaptation window
    DevState* st;
    double* partials;             // [3][4] u64 accumulator slots of the exact parameter-move sums
    unsigned* bar;                // [0] the grid barrier's word
    unsigned long long* flags;    // [2][kMaxGrid] neighbour epoch flags of the sweep
    uint64_t ep0;                 // epoch of the sweep before this launch's first (flags only grow)
    unsigned* ticket;             // last-block counter of single-pass reductions
    double* red;                  // [2][kMaxGrid * kRedStride] per-CTA partials of single-pass reductions
    const double* pdraw;          // [kDrawChunk][NP][2] parameter draws of a resident launch (z, -log u)
    double *S1, *S2, *shift;      // [D*(M+1) + NP] running shifted sums (FP64)
    double *R1, *R2;              // [(D+1)*M] residual sums: eps_{n+1,a} at a*M+n, delta_n at D*M+n-1
    unsigned long long* hist;     // [n_sel][n_bins + 2]
    const int64_t* h_comp;
    const double *h_lo, *h_hi;
    int n_sel, n_bins;
    double* trace;                // [trace_cap][NP] ring of p after each sweep (or null)
    int64_t trace_cap;
    int64_t n_init, n_skip, n_cool;
    double fbeta, f_acc, alpha;
    uint64_t seed;
    uint32_t chain;
    int64_t wait_ns;
    int skip_cta;
    int64_t tile;                 // sites per CTA in the sweep kernel
    unsigned* chk;                // [3][ldx] site visits (even phase, odd phase, parameter-move cache
                                  // writes), then a u64 count of executed parameter moves: counted by
                                  // builds compiled with PIMC_CHECK only
};

// 1 in a build compiled with PIMC_CHECK (the sweep kernels count site visits
// and check site indices), 0 otherwise.
int checked_build();

// Device-side scalars of one HMC trajectory.
struct HmcScalars {
    double A0[3], A1[3];          // action (A, A_o, A_f) at the start and end
    double K0, K1, dH, E, eps;    // kinetic energies, dH, -log u, jittered step
    int oob, accept;
    unsigned long long n_acc, n_traj;
    // parameter momenta by step parity: leapfrog step k writes P_p(k - 1/2)
    // to pp[k & 1] while its CTAs read P_p(k - 3/2) from the other row
    double pp[2][kMaxParams];
};
struct HmcBuffers {
    HmcScalars* hs;
    // [D*(M+1) + NP] each: positions (two buffers), momenta, the trajectory's
    // eps invm, inverse mass; site entries of Q, Q2, P, EM hold a double, or
    // in the FP32-mixed form a float pair hi + lo (parameter entries: double)
    double *Q, *Q2, *P, *EM, *invm;
};
// pdl: launch the kernels after the first with programmatic dependent launch
// (as captured into the trajectory's graph).
cudaError_t launch_hmc_trajectory(int model, int prec, const Ctx& c, const HmcBuffers& b, int n_leap, double eps,
                                  uint64_t seed, bool pdl, cudaStream_t s);

template <class R> constexpr int prec_of();
template <> constexpr int prec_of<double>() { return 0; }
template <> constexpr int prec_of<float>() { return 1; }

// Message returned by pimc_last_error(NULL) on this thread.
void set_thread_error(const char* msg);

// Kernel launchers (model: pimc_model, prec: pimc_precision).
// resident != 0: the resident form where it fits (resident_fits)
cudaError_t launch_sweep(int model, int prec, const Ctx& c, int64_t n_sweeps, int grid, int resident, cudaStream_t s);
// co-resident CTAs on the device of the general (resident = 0) or resident
// (resident = 1, FP32-mixed only; 0 otherwise) sweep kernel
int sweep_max_grid(int model, int prec, int device, int resident);
// whether a launch of `grid` CTAs with tiles of `tile` sites takes the resident form
bool resident_fits(int prec, int64_t tile, int grid);
// One piece of work of a batched launch: chain `chain` alone (size 1), or its
// tile `rank` of `size` equal tiles, which `size` CTAs of the launch run
// together.
struct BatchItem {
    int chain, rank, size, pad;
};
// Many chains in one launch (nt threads per CTA: 128 or 256): CTA b runs
// items[first[b] .. first[b+1]) one after another.  cooperative: some chain
// is split over several CTAs (the launch guarantees they are co-resident).
cudaError_t launch_batch_sweep(int model, int prec, int nt, const Ctx* chains, const int* first,
                               const BatchItem* items, int n_ctas, int64_t n_sweeps, uint64_t seed, bool cooperative,
                               cudaStream_t s);
int batch_ctas_per_sm(int model, int prec, int nt);
cudaError_t launch_init_path(int model, int prec, const Ctx& c, cudaStream_t s);
cudaError_t launch_refresh_cache(int model, int prec, const Ctx& c, cudaStream_t s);
// out: 3 doubles (A, Ao, Af).  X_ext/p_ext: FP64 caller arrays ([D][M+1] dense, [NP]) or null
// for the handle's own state.
cudaError_t launch_action(int model, int prec, const Ctx& c, const double* X_ext, const double* p_ext,
                          double* out, cudaStream_t s);
cudaError_t launch_grad(int model, int prec, const Ctx& c, const double* X_ext, const double* p_ext,
                        double beta, double* gX, double* gp, cudaStream_t s);
cudaError_t launch_site_delta(int model, int prec, const Ctx& c, const double* Xp, double beta,
                              double* dA, cudaStream_t s);
cudaError_t launch_param_delta(int model, int prec, const Ctx& c, int l, double pl_new, double beta,
                               double* out, cudaStream_t s);
// Exact Fix3 sum of n device terms (as FP32 when as_float) into *out (device).
cudaError_t launch_fix_sum(const double* t, int64_t n, int as_float, double* out, cudaStream_t s);
cudaError_t launch_lane_maps(const double* X, const double* I, const double* p, double dt, int64_t n, double* out,
                             unsigned* mismatch, cudaStream_t s);
// dst[i] = (storage type) src[i], i < n.
cudaError_t launch_convert(int prec, const double* src, void* dst, int64_t n, cudaStream_t s);
// Ensemble forecast from the current state: out[e][a][k] (device, FP64).
cudaError_t launch_forecast(int model, int prec, const Ctx& c, int64_t n_steps, const double* I, int n_ens,
                            int noise, uint64_t seed, double* out, cudaStream_t s);
// X conversion between the handle storage and dense FP64 [D][M+1].
cudaError_t launch_path_io(int prec, const Ctx& c, int D, double* dense, int to_state, cudaStream_t s);

}  // namespace pimc
