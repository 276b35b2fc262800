// Host runtime behind the C ABI of include/pimc.h: the handle, its device
// buffers, argument validation, launch geometry, statistics read-back and
// checkpoints.  All arithmetic of the sampler runs in the kernels of sweep.cu
// and ops.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <map>
#include <queue>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pimc.h"
#include "internal.h"

using namespace pimc;

namespace pimc {
// Map-throughput probe (ops.cu): ctas_per_sm (1, 2 or 4) CTAs of 256 threads
// per SM, each thread iterating the HH map `iters` times: FP32 (packed 0),
// FP32 on two packed lanes (1) or FP64 (2); out: n_sm * ctas_per_sm * 256
// floats.
cudaError_t launch_load_refresh(int model, int prec, const Ctx& c, const double* y64, const double* I64, int refresh,
                                cudaStream_t s);
cudaError_t launch_map_rate(int packed, int ctas_per_sm, int n_sm, int64_t iters, float* out, cudaStream_t s);
}  // namespace pimc

struct pimc_handle_s {
    int model = 0, D = 0, NP = 0, prec = 0;
    int scheme = 0, proposal = 0;
    int64_t M = 0, ldx = 0, ldf = 0;
    double dt = 0, Rm = 0, Rf[4] = {0, 0, 0, 0};
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;  // private stream the HMC graph is captured on
    // device buffers (sized for FP64 elements; FP32 storage uses the first half)
    void* X = nullptr;
    void* F[2] = {nullptr, nullptr};
    void* y = nullptr;
    void* I = nullptr;
    void* sig = nullptr;
    uint32_t* acc_win = nullptr;
    DevState* st = nullptr;
    double* partials = nullptr;
    unsigned* bar = nullptr;
    unsigned long long* flags = nullptr;  // neighbour epoch flags [2][kMaxGrid] of the sweep kernel
    uint64_t epoch = 0;                   // sweeps launched so far: the flags' epoch base
    bool resident = false;                // the sweep takes the resident form (one site a thread)
    int form = PIMC_FORM_AUTO;            // forms the sweep may take
    unsigned* ticket = nullptr;
    unsigned* chk = nullptr;          // site-visit counters of checked builds
    double* red = nullptr;
    double* pdraw = nullptr;          // parameter draws of a resident launch
    double *S1 = nullptr, *S2 = nullptr, *shift = nullptr;
    double *R1 = nullptr, *R2 = nullptr;
    unsigned long long* hist = nullptr;
    int64_t* h_comp = nullptr;
    double *h_lo = nullptr, *h_hi = nullptr;
    int n_sel = 0, n_bins = 0;
    double* dense = nullptr;  // D*(M+1) FP64 staging
    double* small = nullptr;  // 16 doubles of results
    HmcBuffers hmc{};         // HMC state (allocated on first use)
    cudaGraphExec_t hmc_exec = nullptr;
    int hmc_leap = -1;
    double hmc_eps = 0.0;
    uint64_t hmc_seed = 0;
    int hmc_prec = -1;
    unsigned ctx_version = 0, hmc_version = ~0u;  // settings captured into the HMC graph
    double* trace = nullptr;  // parameter trace ring [trace_cap][NP]
    int64_t trace_cap = 0;
    double* y64 = nullptr;    // FP64 copies of the data as given (M+1, M)
    double* I64 = nullptr;
    bool have_data = false, have_params = false;
    DevState hs{};
    int64_t n_init = 0, n_skip = 1, n_cool = 0;
    double beta0 = 1.0, fbeta = 1.0, f_acc = 0.4, alpha = 0.0;
    uint32_t chain = 0;
    int64_t wait_ns = 2000000000LL;
    int skip_cta = -1, grid_override = 0;
    int grid = 1;
    int64_t tile = 1;
    std::string err;
};

namespace {

thread_local std::string g_create_error;

int fail(pimc_t h, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_error = buf;
    return code;
}

#define CK(h, call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((h), e_ == cudaErrorMemoryAllocation ? PIMC_ERR_OOM : PIMC_ERR_CUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                            \
    } while (0)

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

size_t esize(pimc_t h) { return h->prec == PIMC_FP64 ? sizeof(double) : sizeof(float); }

Ctx make_ctx(pimc_t h)
{
    Ctx c{};
    c.M = h->M; c.ldx = h->ldx; c.ldf = h->ldf;
    c.scheme = h->scheme; c.proposal = h->proposal;
    c.dt = h->dt; c.Rm = h->Rm;
    for (int a = 0; a < 4; ++a) c.Rf[a] = h->Rf[a];
    c.X = h->X; c.F[0] = h->F[0]; c.F[1] = h->F[1]; c.y = h->y; c.I = h->I; c.sig = h->sig;
    c.acc_win = h->acc_win; c.st = h->st; c.partials = h->partials; c.bar = h->bar; c.flags = h->flags;
    c.ticket = h->ticket; c.red = h->red; c.pdraw = h->pdraw;
    c.S1 = h->S1; c.S2 = h->S2; c.shift = h->shift;
    c.R1 = h->R1; c.R2 = h->R2;
    c.hist = h->hist; c.h_comp = h->h_comp; c.h_lo = h->h_lo; c.h_hi = h->h_hi;
    c.n_sel = h->n_sel; c.n_bins = h->n_bins;
    c.trace = h->trace; c.trace_cap = h->trace_cap;
    c.n_init = h->n_init; c.n_skip = h->n_skip; c.n_cool = h->n_cool;
    c.fbeta = h->fbeta; c.f_acc = h->f_acc; c.alpha = h->alpha;
    c.chain = h->chain; c.wait_ns = h->wait_ns; c.skip_cta = h->skip_cta;
    c.tile = h->tile;
    c.chk = h->chk;
    return c;
}

int pull_state(pimc_t h)
{
    CK(h, cudaMemcpyAsync(&h->hs, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return PIMC_OK;
}

int push_state(pimc_t h)
{
    CK(h, cudaMemcpyAsync(h->st, &h->hs, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return PIMC_OK;
}

// y and I in the storage precision, converted on the device from the FP64
// copies (enqueued on the handle's stream).
int convert_data(pimc_t h)
{
    CK(h, launch_convert(h->prec, h->y64, h->y, h->M + 1, h->stream));
    CK(h, launch_convert(h->prec, h->I64, h->I, h->M, h->stream));
    return PIMC_OK;
}

// Host FP64 arrays -> FP64 device copies -> storage precision.  Asynchronous
// when the host arrays are pinned.
int upload_data(pimc_t h, const double* y, const double* I)
{
    CK(h, cudaMemcpyAsync(h->y64, y, sizeof(double) * (h->M + 1), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->I64, I, sizeof(double) * h->M, cudaMemcpyHostToDevice, h->stream));
    return convert_data(h);
}

// Dense FP64 [D][M+1] host array -> handle storage (X or sig rows), copied on
// the handle's stream (ahead of the work enqueued after it) and complete on
// return.
int put_rows(pimc_t h, void* dst, const double* src)
{
    const int64_t n1 = h->M + 1;
    if (h->prec == PIMC_FP64) {
        CK(h, cudaMemcpy2DAsync(dst, sizeof(double) * h->ldx, src, sizeof(double) * n1, sizeof(double) * n1, h->D,
                                cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    } else {
        std::vector<float> t((size_t)(h->D * n1));
        for (size_t i = 0; i < t.size(); ++i) t[i] = (float)src[i];
        CK(h, cudaMemcpy2DAsync(dst, sizeof(float) * h->ldx, t.data(), sizeof(float) * n1, sizeof(float) * n1, h->D,
                                cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return PIMC_OK;
}

int get_rows(pimc_t h, double* dst, const void* src, int64_t ld, int64_t ncol)
{
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->prec == PIMC_FP64) {
        CK(h, cudaMemcpy2D(dst, sizeof(double) * ncol, src, sizeof(double) * ld, sizeof(double) * ncol, h->D,
                           cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> t((size_t)(h->D * ncol));
        CK(h, cudaMemcpy2D(t.data(), sizeof(float) * ncol, src, sizeof(float) * ld, sizeof(float) * ncol, h->D,
                           cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < t.size(); ++i) dst[i] = (double)t[i];
    }
    return PIMC_OK;
}

int refresh(pimc_t h)
{
    if (!h->have_data || !h->have_params) return PIMC_OK;
    CK(h, launch_refresh_cache(h->model, h->prec, make_ctx(h), h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return PIMC_OK;
}

void choose_grid(pimc_t h)
{
    const int64_t sites = h->M + 1;
    int maxco = sweep_max_grid(h->model, h->prec, h->device, 0);
    if (maxco < 1) maxco = 1;
    if (maxco > kMaxGrid) maxco = kMaxGrid;
    int64_t g;
    if (h->grid_override > 0) {
        g = h->grid_override;
    } else {
        const int64_t by_sm = std::min<int64_t>(h->num_sms, (sites + 63) / 64);
        const int64_t by_threads = (sites + 2 * kSweepBlock - 1) / (2 * kSweepBlock);
        g = std::max<int64_t>(by_sm, by_threads);
    }
    if (g > maxco) g = maxco;
    if (g < 1) g = 1;
    h->tile = (sites + g - 1) / g;
    // tiles of even length when tiled: every CTA's first site is even, so a
    // tile's halo sites change in fixed phases of the sweep
    if (g > 1) h->tile += h->tile & 1;
    h->grid = (int)((sites + h->tile - 1) / h->tile);
    h->resident = h->form == PIMC_FORM_AUTO && resident_fits(h->prec, h->tile, h->grid) &&
                  h->grid <= sweep_max_grid(h->model, h->prec, h->device, 1);
}

int check_finite(const double* v, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return 0;
    return 1;
}

void free_all(pimc_t h)
{
    void* bufs[] = {h->X, h->F[0], h->F[1], h->y, h->I, h->sig, h->acc_win, h->st, h->partials, h->bar, h->flags,
                    h->ticket, h->chk, h->red, h->pdraw, h->S1, h->S2, h->shift, h->hist, h->h_comp, h->h_lo, h->h_hi,
                    h->dense, h->small, h->y64, h->I64, h->trace, h->R1, h->R2, h->hmc.hs, h->hmc.Q, h->hmc.P,
                    h->hmc.Q2, h->hmc.EM, h->hmc.invm};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (h->hmc_exec) cudaGraphExecDestroy(h->hmc_exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
}

// clear statistics, counters and windows (sweep counter and beta follow the
// schedule); stream-ordered: the handle's stream does not wait for the legacy
// default stream
int reset_stats(pimc_t h)
{
    const int64_t nc = (int64_t)h->D * (h->M + 1) + h->NP;
    cudaStream_t st = h->stream;
    CK(h, cudaMemsetAsync(h->S1, 0, sizeof(double) * nc, st));
    CK(h, cudaMemsetAsync(h->S2, 0, sizeof(double) * nc, st));
    CK(h, cudaMemsetAsync(h->shift, 0, sizeof(double) * nc, st));
    CK(h, cudaMemsetAsync(h->acc_win, 0, sizeof(uint32_t) * h->ldx, st));
    CK(h, cudaMemsetAsync(h->R1, 0, sizeof(double) * (h->D + 1) * h->M, st));
    CK(h, cudaMemsetAsync(h->R2, 0, sizeof(double) * (h->D + 1) * h->M, st));
    if (h->hist) CK(h, cudaMemsetAsync(h->hist, 0, sizeof(unsigned long long) * kMaxSel * (kMaxBins + 2), st));
    return PIMC_OK;
}

}  // namespace

void pimc::set_thread_error(const char* msg) { g_create_error = msg; }

extern "C" {

int pimc_create(pimc_t* out, int model, int64_t M, int D, int L, double dt, const double* Rm, const double* Rf)
{
    if (!out) return fail(nullptr, PIMC_ERR_ARG, "out is NULL");
    *out = nullptr;
    int Dm, NP;
    switch (model) {
    case PIMC_MODEL_HH: Dm = 4; NP = 7; break;
    case PIMC_MODEL_LINGAUSS: Dm = 2; NP = 1; break;
    case PIMC_MODEL_TOY1D: Dm = 1; NP = 1; break;
    case PIMC_MODEL_HH_PAPER: Dm = 4; NP = 7; break;
    default: return fail(nullptr, PIMC_ERR_ARG, "unknown model %d", model);
    }
    if (M < 1 || M > (int64_t)1 << 31) return fail(nullptr, PIMC_ERR_ARG, "M must be in [1, 2^31], got %lld", (long long)M);
    if (D != Dm) return fail(nullptr, PIMC_ERR_ARG, "model %d has D = %d, got %d", model, Dm, D);
    if (L != 1) return fail(nullptr, PIMC_ERR_ARG, "only L = 1 (h(x) = x_0) is supported, got %d", L);
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, PIMC_ERR_ARG, "dt must be finite and > 0");
    if (!Rm || !(*Rm > 0.0) || !std::isfinite(*Rm)) return fail(nullptr, PIMC_ERR_ARG, "Rm must be finite and > 0");
    if (!Rf) return fail(nullptr, PIMC_ERR_ARG, "Rf is NULL");
    for (int a = 0; a < D; ++a)
        if (!(Rf[a] >= 0.0) || !std::isfinite(Rf[a])) return fail(nullptr, PIMC_ERR_ARG, "Rf[%d] must be finite and >= 0", a);

    pimc_t h = new pimc_handle_s();
    h->model = model; h->D = D; h->NP = NP; h->M = M; h->dt = dt; h->Rm = *Rm;
    for (int a = 0; a < D; ++a) h->Rf[a] = Rf[a];
    h->ldx = round_up(M + 1, 64);
    h->ldf = round_up(M + 1, 64);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        int r = fail(nullptr, PIMC_ERR_CUDA, "device setup: %s", cudaGetErrorString(e));
        delete h;
        return r;
    }
    h->own_stream = true;
    const int64_t nc = (int64_t)D * (M + 1) + NP;
    struct { void** p; size_t bytes; } allocs[] = {
        {&h->X, sizeof(double) * D * h->ldx},
        {&h->F[0], sizeof(double) * D * h->ldf},
        {&h->F[1], sizeof(double) * D * h->ldf},
        {&h->y, sizeof(double) * h->ldx},
        {&h->I, sizeof(double) * h->ldf},
        {&h->sig, sizeof(double) * D * h->ldx},
        {(void**)&h->acc_win, sizeof(uint32_t) * h->ldx},
        {(void**)&h->st, sizeof(DevState)},
        {(void**)&h->partials, sizeof(double) * 2 * kMaxGrid},
        {(void**)&h->bar, sizeof(unsigned) * 4},
        {(void**)&h->flags, sizeof(unsigned long long) * 2 * kMaxGrid},
        {(void**)&h->ticket, sizeof(unsigned) * 4},
        {(void**)&h->chk, sizeof(unsigned) * (3 * h->ldx + 2)},
        {(void**)&h->red, sizeof(double) * 2 * kRedStride * kMaxGrid},
        {(void**)&h->pdraw, sizeof(double) * 2 * kMaxParams * kDrawChunk},
        {(void**)&h->S1, sizeof(double) * nc},
        {(void**)&h->S2, sizeof(double) * nc},
        {(void**)&h->shift, sizeof(double) * nc},
        {(void**)&h->dense, sizeof(double) * D * (M + 1)},
        {(void**)&h->small, sizeof(double) * 16},
        {(void**)&h->R1, sizeof(double) * (D + 1) * M},
        {(void**)&h->R2, sizeof(double) * (D + 1) * M},
        {(void**)&h->y64, sizeof(double) * (M + 1)},
        {(void**)&h->I64, sizeof(double) * M},
    };
    for (auto& a : allocs) {
        e = cudaMalloc(a.p, a.bytes);
        if (e != cudaSuccess) {
            int r = fail(nullptr, e == cudaErrorMemoryAllocation ? PIMC_ERR_OOM : PIMC_ERR_CUDA,
                         "cudaMalloc(%zu): %s", a.bytes, cudaGetErrorString(e));
            free_all(h);
            cudaStreamDestroy(h->stream);
            delete h;
            return r;
        }
    }
    // zeroed on the handle's stream, ahead of everything launched on it
    cudaMemsetAsync(h->bar, 0, sizeof(unsigned) * 4, h->stream);
    cudaMemsetAsync(h->flags, 0, sizeof(unsigned long long) * 2 * kMaxGrid, h->stream);
    cudaMemsetAsync(h->ticket, 0, sizeof(unsigned) * 4, h->stream);
    cudaMemsetAsync(h->chk, 0, sizeof(unsigned) * (3 * h->ldx + 2), h->stream);
    cudaMemsetAsync(h->X, 0, sizeof(double) * D * h->ldx, h->stream);
    cudaMemsetAsync(h->F[0], 0, sizeof(double) * D * h->ldf, h->stream);
    cudaMemsetAsync(h->F[1], 0, sizeof(double) * D * h->ldf, h->stream);
    cudaMemsetAsync(h->sig, 0, sizeof(double) * D * h->ldx, h->stream);
    h->hs = DevState{};
    h->hs.beta = 1.0;
    for (int l = 0; l < kMaxParams; ++l) { h->hs.lo[l] = -INFINITY; h->hs.hi[l] = INFINITY; }
    cudaMemsetAsync(h->y64, 0, sizeof(double) * (M + 1), h->stream);
    cudaMemsetAsync(h->I64, 0, sizeof(double) * M, h->stream);
    int r = push_state(h);
    if (r == PIMC_OK) r = reset_stats(h);
    if (r != PIMC_OK) {
        g_create_error = h->err;
        pimc_destroy(h);
        return r;
    }
    choose_grid(h);
    *out = h;
    return PIMC_OK;
}

int pimc_destroy(pimc_t h)
{
    if (!h) return PIMC_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return PIMC_OK;
}

const char* pimc_last_error(pimc_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int pimc_set_stream(pimc_t h, void* stream)
{
    if (!h) return PIMC_ERR_ARG;
    h->ctx_version++;
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->own_stream) cudaStreamDestroy(h->stream);
    h->own_stream = false;
    h->stream = (cudaStream_t)stream;
    return PIMC_OK;
}

int pimc_set_precision(pimc_t h, int precision)
{
    if (!h) return PIMC_ERR_ARG;
    if (precision != PIMC_FP64 && precision != PIMC_FP32_MIXED)
        return fail(h, PIMC_ERR_ARG, "unknown precision %d", precision);
    if (precision == h->prec) return PIMC_OK;
    h->ctx_version++;
    const int64_t nd = (int64_t)h->D * (h->M + 1);
    std::vector<double> X(nd), S(nd);
    int r = get_rows(h, X.data(), h->X, h->ldx, h->M + 1);
    if (r == PIMC_OK) r = get_rows(h, S.data(), h->sig, h->ldx, h->M + 1);
    if (r != PIMC_OK) return r;
    h->prec = precision;
    if ((r = put_rows(h, h->X, X.data())) != PIMC_OK) return r;
    if ((r = put_rows(h, h->sig, S.data())) != PIMC_OK) return r;
    if (h->have_data && (r = convert_data(h)) != PIMC_OK) return r;
    choose_grid(h);
    return refresh(h);
}

int pimc_set_scheme(pimc_t h, int scheme)
{
    if (!h) return PIMC_ERR_ARG;
    if (scheme != PIMC_SCHEME_RK4 && scheme != PIMC_SCHEME_TRAPEZOID) return fail(h, PIMC_ERR_ARG, "unknown scheme %d", scheme);
    h->scheme = scheme;
    h->ctx_version++;
    return refresh(h);
}

int pimc_set_proposal(pimc_t h, int kind)
{
    if (!h) return PIMC_ERR_ARG;
    if (kind != PIMC_PROPOSAL_GAUSS && kind != PIMC_PROPOSAL_UNIFORM) return fail(h, PIMC_ERR_ARG, "unknown proposal %d", kind);
    h->proposal = kind;
    h->ctx_version++;
    return PIMC_OK;
}

int pimc_set_data(pimc_t h, const double* y, const double* I_inj)
{
    if (!h) return PIMC_ERR_ARG;
    if (!y || !I_inj) return fail(h, PIMC_ERR_ARG, "y or I_inj is NULL");
    if (!check_finite(y, h->M + 1)) return fail(h, PIMC_ERR_ARG, "y has non-finite values");
    if (!check_finite(I_inj, h->M)) return fail(h, PIMC_ERR_ARG, "I_inj has non-finite values");
    int r = upload_data(h, y, I_inj);
    if (r != PIMC_OK) return r;
    h->have_data = true;
    CK(h, launch_init_path(h->model, h->prec, make_ctx(h), h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return refresh(h);
}

int pimc_load_data(pimc_t h, const double* y, const double* I_inj)
{
    if (!h) return PIMC_ERR_ARG;
    if (!h->have_data) return fail(h, PIMC_ERR_STATE, "pimc_load_data before pimc_set_data");
    if (!y || !I_inj) return fail(h, PIMC_ERR_ARG, "y or I_inj is NULL");
    if (!check_finite(y, h->M + 1)) return fail(h, PIMC_ERR_ARG, "y has non-finite values");
    if (!check_finite(I_inj, h->M)) return fail(h, PIMC_ERR_ARG, "I_inj has non-finite values");
    CK(h, cudaMemcpyAsync(h->y64, y, sizeof(double) * (h->M + 1), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->I64, I_inj, sizeof(double) * h->M, cudaMemcpyHostToDevice, h->stream));
    // conversion and cache refresh in one launch
    CK(h, launch_load_refresh(h->model, h->prec, make_ctx(h), h->y64, h->I64, h->have_params ? 1 : 0, h->stream));
    return PIMC_OK;
}

int pimc_set_params(pimc_t h, const double* p, const double* lo, const double* hi, const uint8_t* free_mask, int Np)
{
    if (!h) return PIMC_ERR_ARG;
    if (Np != h->NP) return fail(h, PIMC_ERR_ARG, "model has Np = %d, got %d", h->NP, Np);
    if (!p) return fail(h, PIMC_ERR_ARG, "p is NULL");
    int r = pull_state(h);
    if (r != PIMC_OK) return r;
    unsigned mask = 0;
    for (int l = 0; l < Np; ++l) {
        const double L = lo ? lo[l] : -INFINITY, H = hi ? hi[l] : INFINITY;
        const int fr = free_mask ? (free_mask[l] != 0) : 0;
        if (!std::isfinite(p[l])) return fail(h, PIMC_ERR_ARG, "p[%d] is not finite", l);
        if (std::isnan(L) || std::isnan(H) || L > H) return fail(h, PIMC_ERR_ARG, "bad bounds for p[%d]", l);
        if (fr && !(p[l] >= L && p[l] <= H)) return fail(h, PIMC_ERR_ARG, "p[%d] outside its prior box", l);
        h->hs.p[l] = p[l]; h->hs.lo[l] = L; h->hs.hi[l] = H;
        if (fr) mask |= 1u << l;
    }
    h->hs.free_mask = mask;
    if ((r = push_state(h)) != PIMC_OK) return r;
    h->have_params = true;
    return refresh(h);
}

int pimc_set_path(pimc_t h, const double* X)
{
    if (!h) return PIMC_ERR_ARG;
    if (!X) {
        if (!h->have_data) return fail(h, PIMC_ERR_STATE, "default path needs pimc_set_data first");
        CK(h, launch_init_path(h->model, h->prec, make_ctx(h), h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        return refresh(h);
    }
    if (!check_finite(X, (int64_t)h->D * (h->M + 1))) return fail(h, PIMC_ERR_ARG, "X has non-finite values");
    int r = put_rows(h, h->X, X);
    if (r != PIMC_OK) return r;
    return refresh(h);
}

int pimc_set_steps(pimc_t h, const double* sigma_x, int per_site, const double* sigma_p)
{
    if (!h) return PIMC_ERR_ARG;
    const int64_t n1 = h->M + 1, nd = (int64_t)h->D * n1;
    if (sigma_x) {
        std::vector<double> S(nd);
        for (int a = 0; a < h->D; ++a)
            for (int64_t n = 0; n < n1; ++n) S[a * n1 + n] = per_site ? sigma_x[a * n1 + n] : sigma_x[a];
        for (double v : S)
            if (!(v >= 0.0) || !std::isfinite(v)) return fail(h, PIMC_ERR_ARG, "sigma_x must be finite and >= 0");
        int r = put_rows(h, h->sig, S.data());
        if (r != PIMC_OK) return r;
    }
    if (sigma_p) {
        int r = pull_state(h);
        if (r != PIMC_OK) return r;
        for (int l = 0; l < h->NP; ++l) {
            if (!(sigma_p[l] >= 0.0) || !std::isfinite(sigma_p[l])) return fail(h, PIMC_ERR_ARG, "sigma_p must be finite and >= 0");
            h->hs.sigp[l] = sigma_p[l];
        }
        return push_state(h);
    }
    return PIMC_OK;
}

int pimc_set_schedule(pimc_t h, int64_t n_init, int64_t n_skip, double beta0, int64_t n_cool, double f_acc, double alpha)
{
    if (!h) return PIMC_ERR_ARG;
    h->ctx_version++;
    if (n_skip < 1 || n_init < 0 || n_cool < 0 || !(beta0 > 0.0) || beta0 > 1.0 || !std::isfinite(f_acc) ||
        !std::isfinite(alpha))
        return fail(h, PIMC_ERR_ARG, "bad schedule");
    h->n_init = n_init; h->n_skip = n_skip; h->n_cool = n_cool; h->beta0 = beta0;
    h->f_acc = f_acc; h->alpha = alpha;
    h->fbeta = n_cool > 0 ? std::pow(1.0 / beta0, 1.0 / (double)n_cool) : 1.0;
    int r = pull_state(h);
    if (r != PIMC_OK) return r;
    h->hs.sweep = 0;
    h->hs.J = 0;
    h->hs.beta = n_cool > 0 ? beta0 : 1.0;
    for (int l = 0; l < kMaxParams; ++l) { h->hs.accp_win[l] = 0; h->hs.par_acc[l] = 0; h->hs.par_prop[l] = 0; }
    h->hs.site_acc[0] = h->hs.site_acc[1] = h->hs.site_prop[0] = h->hs.site_prop[1] = h->hs.nonfinite = 0;
    if ((r = push_state(h)) != PIMC_OK) return r;
    return reset_stats(h);
}

int pimc_set_chain(pimc_t h, uint32_t chain)
{
    if (!h) return PIMC_ERR_ARG;
    h->ctx_version++;
    h->chain = chain;
    return PIMC_OK;
}

int pimc_sweep(pimc_t h, int64_t n_sweeps, uint64_t seed)
{
    if (!h) return PIMC_ERR_ARG;
    if (!h->have_data || !h->have_params) return fail(h, PIMC_ERR_STATE, "pimc_sweep before pimc_set_data/pimc_set_params");
    if (n_sweeps < 0) return fail(h, PIMC_ERR_ARG, "n_sweeps < 0");
    Ctx c = make_ctx(h);
    c.seed = seed;
    const int64_t chunk = kDrawChunk;  // bound the duration of one launch
    for (int64_t done = 0; done < n_sweeps; done += chunk) {
        const int64_t k = std::min<int64_t>(chunk, n_sweeps - done);
        c.ep0 = h->epoch;
        CK(h, launch_sweep(h->model, h->prec, c, k, h->grid, h->resident ? 1 : 0, h->stream));
        h->epoch += (uint64_t)k;
    }
    return PIMC_OK;
}

int pimc_sync(pimc_t h)
{
    if (!h) return PIMC_ERR_ARG;
    int r = pull_state(h);
    if (r != PIMC_OK) return r;
    if (h->hs.status & kStatusTimeout) {
        h->hs.status = 0;
        h->hs.abort = 0;
        CK(h, cudaMemsetAsync(h->bar, 0, sizeof(unsigned) * 4, h->stream));
        if ((r = push_state(h)) != PIMC_OK) return r;
        return fail(h, PIMC_ERR_TIMEOUT, "a bounded grid-barrier wait expired; the sweep launch returned early");
    }
    return PIMC_OK;
}

int pimc_action(pimc_t h, double* A_out, double* Ao_out, double* Af_out)
{
    if (!h) return PIMC_ERR_ARG;
    if (!h->have_data || !h->have_params) return fail(h, PIMC_ERR_STATE, "pimc_action before data/params");
    CK(h, launch_action(h->model, h->prec, make_ctx(h), nullptr, nullptr, h->small, h->stream));
    double r[3];
    CK(h, cudaMemcpyAsync(r, h->small, sizeof r, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (A_out) *A_out = r[0];
    if (Ao_out) *Ao_out = r[1];
    if (Af_out) *Af_out = r[2];
    return PIMC_OK;
}

int pimc_grad(pimc_t h, double beta, double* gX, double* gp)
{
    if (!h) return PIMC_ERR_ARG;
    if (!h->have_data || !h->have_params) return fail(h, PIMC_ERR_STATE, "pimc_grad before data/params");
    if (!gX || !gp) return fail(h, PIMC_ERR_ARG, "NULL output");
    CK(h, launch_grad(h->model, h->prec, make_ctx(h), nullptr, nullptr, beta, h->dense, h->small, h->stream));
    CK(h, cudaMemcpyAsync(gX, h->dense, sizeof(double) * h->D * (h->M + 1), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(gp, h->small, sizeof(double) * h->NP, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return PIMC_OK;
}

int pimc_action_dev(pimc_t h, const double* X_dev, const double* p_dev, double* out_dev, void* stream)
{
    if (!h) return PIMC_ERR_ARG;
    if (!h->have_data) return fail(h, PIMC_ERR_STATE, "pimc_action_dev before pimc_set_data");
    if (!X_dev || !p_dev || !out_dev) return fail(h, PIMC_ERR_ARG, "NULL device pointer");
    CK(h, launch_action(h->model, h->prec, make_ctx(h), X_dev, p_dev, out_dev, (cudaStream_t)stream));
    return PIMC_OK;
}

int pimc_grad_dev(pimc_t h, const double* X_dev, const double* p_dev, double beta, double* gX_dev, double* gp_dev,
                  void* stream)
{
    if (!h) return PIMC_ERR_ARG;
    if (!h->have_data) return fail(h, PIMC_ERR_STATE, "pimc_grad_dev before pimc_set_data");
    if (!X_dev || !p_dev || !gX_dev || !gp_dev) return fail(h, PIMC_ERR_ARG, "NULL device pointer");
    CK(h, launch_grad(h->model, h->prec, make_ctx(h), X_dev, p_dev, beta, gX_dev, gp_dev, (cudaStream_t)stream));
    return PIMC_OK;
}

int pimc_site_delta(pimc_t h, const double* Xp, double beta, double* dA_out)
{
    if (!h) return PIMC_ERR_ARG;
    if (!h->have_data || !h->have_params) return fail(h, PIMC_ERR_STATE, "pimc_site_delta before data/params");
    if (!Xp || !dA_out) return fail(h, PIMC_ERR_ARG, "NULL argument");
    const int64_t nd = (int64_t)h->D * (h->M + 1);
    double* dA = nullptr;
    CK(h, cudaMalloc(&dA, sizeof(double) * (h->M + 1)));
    cudaError_t e = cudaMemcpyAsync(h->dense, Xp, sizeof(double) * nd, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_site_delta(h->model, h->prec, make_ctx(h), h->dense, beta, dA, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dA_out, dA, sizeof(double) * (h->M + 1), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dA);
    CK(h, e);
    return PIMC_OK;
}

int pimc_param_delta(pimc_t h, int l, double pl_new, double beta, double* dA_out)
{
    if (!h) return PIMC_ERR_ARG;
    if (!h->have_data || !h->have_params) return fail(h, PIMC_ERR_STATE, "pimc_param_delta before data/params");
    if (l < 0 || l >= h->NP || !dA_out) return fail(h, PIMC_ERR_ARG, "bad parameter index or NULL output");
    CK(h, launch_param_delta(h->model, h->prec, make_ctx(h), l, pl_new, beta, h->small, h->stream));
    CK(h, cudaMemcpyAsync(dA_out, h->small, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return PIMC_OK;
}

int pimc_moments(pimc_t h, double* mean, double* var, int64_t* n_samples)
{
    if (!h) return PIMC_ERR_ARG;
    int r = pull_state(h);
    if (r != PIMC_OK) return r;
    const int64_t nc = (int64_t)h->D * (h->M + 1) + h->NP;
    std::vector<double> S1(nc), S2(nc), sh(nc);
    CK(h, cudaMemcpy(S1.data(), h->S1, sizeof(double) * nc, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(S2.data(), h->S2, sizeof(double) * nc, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(sh.data(), h->shift, sizeof(double) * nc, cudaMemcpyDeviceToHost));
    const double J = (double)h->hs.J;
    for (int64_t c = 0; c < nc; ++c) {
        if (mean) mean[c] = h->hs.J > 0 ? sh[c] + S1[c] / J : NAN;
        if (var) var[c] = h->hs.J > 1 ? (S2[c] - S1[c] * S1[c] / J) / (J - 1.0) : NAN;
    }
    if (n_samples) *n_samples = h->hs.J;
    return PIMC_OK;
}

int pimc_residual_moments(pimc_t h, double* mean, double* var, int64_t* n_samples)
{
    if (!h) return PIMC_ERR_ARG;
    int r = pull_state(h);
    if (r != PIMC_OK) return r;
    const int64_t nr = (int64_t)(h->D + 1) * h->M;
    std::vector<double> R1(nr), R2(nr);
    CK(h, cudaMemcpy(R1.data(), h->R1, sizeof(double) * nr, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(R2.data(), h->R2, sizeof(double) * nr, cudaMemcpyDeviceToHost));
    const double J = (double)h->hs.J;
    for (int64_t i = 0; i < nr; ++i) {
        if (mean) mean[i] = h->hs.J > 0 ? R1[i] / J : NAN;
        if (var) var[i] = h->hs.J > 1 ? (R2[i] - R1[i] * R1[i] / J) / (J - 1.0) : NAN;
    }
    if (n_samples) *n_samples = h->hs.J;
    return PIMC_OK;
}

int pimc_forecast(pimc_t h, int64_t n_steps, const double* I_future, int n_ens, int noise, uint64_t seed,
                  double* out)
{
    if (!h) return PIMC_ERR_ARG;
    if (!h->have_data || !h->have_params) return fail(h, PIMC_ERR_STATE, "pimc_forecast before data/params");
    if (n_steps < 0 || n_ens < 1 || !out || (n_steps > 0 && !I_future))
        return fail(h, PIMC_ERR_ARG, "bad forecast arguments");
    if (h->scheme != PIMC_SCHEME_RK4) return fail(h, PIMC_ERR_STATE, "forecasts integrate the explicit RK4 map (scheme RK4)");
    if (!check_finite(I_future, n_steps)) return fail(h, PIMC_ERR_ARG, "I_future has non-finite values");
    const size_t nout = (size_t)n_ens * h->D * (n_steps + 1);
    double *dI = nullptr, *dout = nullptr;
    CK(h, cudaMalloc(&dI, sizeof(double) * std::max<int64_t>(n_steps, 1)));
    cudaError_t e = cudaMalloc(&dout, sizeof(double) * nout);
    if (e == cudaSuccess && n_steps > 0)
        e = cudaMemcpyAsync(dI, I_future, sizeof(double) * n_steps, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_forecast(h->model, h->prec, make_ctx(h), n_steps, dI, n_ens, noise, seed, dout, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(double) * nout, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dI);
    if (dout) cudaFree(dout);
    CK(h, e);
    return PIMC_OK;
}

int pimc_set_histograms(pimc_t h, int n_sel, const int64_t* comp_index, const double* lo, const double* hi, int n_bins)
{
    if (!h) return PIMC_ERR_ARG;
    h->ctx_version++;
    if (n_sel < 1 || n_sel > kMaxSel || n_bins < 1 || n_bins > kMaxBins || !comp_index || !lo || !hi)
        return fail(h, PIMC_ERR_ARG, "bad histogram configuration");
    const int64_t nc = (int64_t)h->D * (h->M + 1) + h->NP;
    for (int k = 0; k < n_sel; ++k) {
        if (comp_index[k] < 0 || comp_index[k] >= nc) return fail(h, PIMC_ERR_ARG, "component index out of range");
        if (!(lo[k] < hi[k]) || !std::isfinite(lo[k]) || !std::isfinite(hi[k]))
            return fail(h, PIMC_ERR_ARG, "histogram range must be finite with lo < hi");
    }
    CK(h, cudaStreamSynchronize(h->stream));
    if (!h->hist) {
        CK(h, cudaMalloc(&h->hist, sizeof(unsigned long long) * kMaxSel * (kMaxBins + 2)));
        CK(h, cudaMalloc(&h->h_comp, sizeof(int64_t) * kMaxSel));
        CK(h, cudaMalloc(&h->h_lo, sizeof(double) * kMaxSel));
        CK(h, cudaMalloc(&h->h_hi, sizeof(double) * kMaxSel));
    }
    CK(h, cudaMemsetAsync(h->hist, 0, sizeof(unsigned long long) * kMaxSel * (kMaxBins + 2), h->stream));
    CK(h, cudaMemcpyAsync(h->h_comp, comp_index, sizeof(int64_t) * n_sel, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->h_lo, lo, sizeof(double) * n_sel, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->h_hi, hi, sizeof(double) * n_sel, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));  // the caller's arrays are read before returning
    h->n_sel = n_sel;
    h->n_bins = n_bins;
    return PIMC_OK;
}

int pimc_histograms(pimc_t h, uint64_t* counts)
{
    if (!h) return PIMC_ERR_ARG;
    if (!h->hist || h->n_sel == 0) return fail(h, PIMC_ERR_STATE, "no histograms configured");
    if (!counts) return fail(h, PIMC_ERR_ARG, "counts is NULL");
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(counts, h->hist, sizeof(uint64_t) * h->n_sel * (h->n_bins + 2), cudaMemcpyDeviceToHost));
    return PIMC_OK;
}

int pimc_hmc(pimc_t h, int64_t n_traj, int n_leap, double eps, const double* inv_mass, uint64_t seed,
             int64_t* n_accepted)
{
    if (!h) return PIMC_ERR_ARG;
    if (!h->have_data || !h->have_params) return fail(h, PIMC_ERR_STATE, "pimc_hmc before data/params");
    if (n_traj < 0 || n_leap < 1 || n_leap > 100000 || !(eps > 0.0) || !std::isfinite(eps))
        return fail(h, PIMC_ERR_ARG, "bad HMC arguments (n_traj >= 0, 1 <= n_leap, eps > 0)");
    const int64_t nq = (int64_t)h->D * (h->M + 1) + h->NP;
    if (!h->hmc.hs) {
        CK(h, cudaMalloc(&h->hmc.hs, sizeof(HmcScalars)));
        CK(h, cudaMalloc(&h->hmc.Q, sizeof(double) * nq));
        CK(h, cudaMalloc(&h->hmc.P, sizeof(double) * nq));
        CK(h, cudaMalloc(&h->hmc.Q2, sizeof(double) * nq));
        CK(h, cudaMalloc(&h->hmc.EM, sizeof(double) * nq));
        CK(h, cudaMalloc(&h->hmc.invm, sizeof(double) * nq));
        CK(h, cudaMemsetAsync(h->hmc.hs, 0, sizeof(HmcScalars), h->stream));
    }
    {
        std::vector<double> im((size_t)nq, 1.0);
        if (inv_mass) {
            for (int64_t j = 0; j < nq; ++j) {
                if (!(inv_mass[j] >= 0.0) || !std::isfinite(inv_mass[j]))
                    return fail(h, PIMC_ERR_ARG, "inv_mass must be finite and >= 0");
                im[j] = inv_mass[j];
            }
        }
        CK(h, cudaMemcpyAsync(h->hmc.invm, im.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    unsigned long long acc0 = 0;
    if (n_accepted) {
        HmcScalars hs;
        CK(h, cudaMemcpyAsync(&hs, h->hmc.hs, sizeof hs, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        acc0 = hs.n_acc;
    }
    // one trajectory = a fixed launch sequence: capture it once as a CUDA graph
    // (re-captured when n_leap, eps, seed or the precision change)
    if (!h->hmc_exec || h->hmc_leap != n_leap || h->hmc_eps != eps || h->hmc_seed != seed || h->hmc_prec != h->prec ||
        h->hmc_version != h->ctx_version) {
        if (h->hmc_exec) {
            cudaGraphExecDestroy(h->hmc_exec);
            h->hmc_exec = nullptr;
        }
        // captured on a private stream (the legacy default stream cannot be
        // captured) and launched on the handle's stream, whichever that is
        if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e =
            launch_hmc_trajectory(h->model, h->prec, make_ctx(h), h->hmc, n_leap, eps, seed, true, h->cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->hmc_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        CK(h, e);
        h->hmc_leap = n_leap;
        h->hmc_eps = eps;
        h->hmc_seed = seed;
        h->hmc_prec = h->prec;
        h->hmc_version = h->ctx_version;
    }
    for (int64_t t = 0; t < n_traj; ++t) CK(h, cudaGraphLaunch(h->hmc_exec, h->stream));
    if (n_accepted) {
        HmcScalars hs;
        CK(h, cudaMemcpyAsync(&hs, h->hmc.hs, sizeof hs, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        *n_accepted = (int64_t)(hs.n_acc - acc0);
        return pimc_sync(h);  // sticky status of the handle (a timed-out wait of an earlier launch)
    }
    return PIMC_OK;
}

int pimc_set_param_trace(pimc_t h, int64_t cap)
{
    if (!h) return PIMC_ERR_ARG;
    h->ctx_version++;
    if (cap < 0 || cap > ((int64_t)1 << 28)) return fail(h, PIMC_ERR_ARG, "trace capacity must be in [0, 2^28]");
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->trace) {
        CK(h, cudaFree(h->trace));
        h->trace = nullptr;
    }
    h->trace_cap = 0;
    if (cap > 0) {
        CK(h, cudaMalloc(&h->trace, sizeof(double) * (size_t)cap * h->NP));
        h->trace_cap = cap;
    }
    int r = pull_state(h);
    if (r != PIMC_OK) return r;
    h->hs.tr_n = 0;
    return push_state(h);
}

int pimc_param_trace(pimc_t h, double* out, int64_t cap, int64_t* n_written)
{
    if (!h) return PIMC_ERR_ARG;
    if (!h->trace) return fail(h, PIMC_ERR_STATE, "no parameter trace configured");
    int r = pull_state(h);
    if (r != PIMC_OK) return r;
    const int64_t total = h->hs.tr_n;
    int64_t k = std::min<int64_t>(total, h->trace_cap);
    if (out) k = std::min<int64_t>(k, cap);
    if (n_written) *n_written = k;
    if (!out || k == 0) return PIMC_OK;
    // the last k entries in chronological order: ring slots (total-k .. total-1) mod cap
    std::vector<double> ring((size_t)h->trace_cap * h->NP);
    CK(h, cudaMemcpy(ring.data(), h->trace, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < k; ++i) {
        const int64_t slot = (total - k + i) % h->trace_cap;
        memcpy(out + i * h->NP, &ring[(size_t)slot * h->NP], sizeof(double) * h->NP);
    }
    return PIMC_OK;
}

int pimc_histogram_shape(pimc_t h, int* n_sel, int* n_bins)
{
    if (!h) return PIMC_ERR_ARG;
    if (n_sel) *n_sel = h->n_sel;
    if (n_bins) *n_bins = h->n_bins;
    return PIMC_OK;
}

int pimc_get_state(pimc_t h, double* X, double* p)
{
    if (!h) return PIMC_ERR_ARG;
    if (X) {
        int r = get_rows(h, X, h->X, h->ldx, h->M + 1);
        if (r != PIMC_OK) return r;
    }
    if (p) {
        int r = pull_state(h);
        if (r != PIMC_OK) return r;
        for (int l = 0; l < h->NP; ++l) p[l] = h->hs.p[l];
    }
    return PIMC_OK;
}

int pimc_params_async(pimc_t h, double* p_host)
{
    if (!h || !p_host) return fail(h, PIMC_ERR_ARG, "pimc_params_async: NULL argument");
    const double* src = (const double*)((const char*)h->st + offsetof(DevState, p));
    CK(h, cudaMemcpyAsync(p_host, src, sizeof(double) * h->NP, cudaMemcpyDeviceToHost, h->stream));
    return PIMC_OK;
}

int pimc_get_steps(pimc_t h, double* sigma_x, double* sigma_p)
{
    if (!h) return PIMC_ERR_ARG;
    if (sigma_x) {
        int r = get_rows(h, sigma_x, h->sig, h->ldx, h->M + 1);
        if (r != PIMC_OK) return r;
    }
    if (sigma_p) {
        int r = pull_state(h);
        if (r != PIMC_OK) return r;
        for (int l = 0; l < h->NP; ++l) sigma_p[l] = h->hs.sigp[l];
    }
    return PIMC_OK;
}

int pimc_get_sweep(pimc_t h, int64_t* sweep, double* beta)
{
    if (!h) return PIMC_ERR_ARG;
    int r = pull_state(h);
    if (r != PIMC_OK) return r;
    if (sweep) *sweep = h->hs.sweep;
    if (beta) *beta = h->hs.beta;
    return PIMC_OK;
}

int pimc_accept_stats(pimc_t h, uint64_t* site_acc, uint64_t* site_prop, uint64_t* par_acc, uint64_t* par_prop)
{
    if (!h) return PIMC_ERR_ARG;
    int r = pull_state(h);
    if (r != PIMC_OK) return r;
    for (int k = 0; k < 2; ++k) {
        if (site_acc) site_acc[k] = h->hs.site_acc[k];
        if (site_prop) site_prop[k] = h->hs.site_prop[k];
    }
    for (int l = 0; l < h->NP; ++l) {
        if (par_acc) par_acc[l] = h->hs.par_acc[l];
        if (par_prop) par_prop[l] = h->hs.par_prop[l];
    }
    return PIMC_OK;
}

int pimc_launch_info(pimc_t h, int* grid, int* block)
{
    if (!h) return PIMC_ERR_ARG;
    if (grid) *grid = h->grid;
    if (block) *block = kSweepBlock;
    return PIMC_OK;
}

int pimc_sweep_form(pimc_t h, int* resident)
{
    if (!h || !resident) return PIMC_ERR_ARG;
    *resident = h->resident ? 1 : 0;
    return PIMC_OK;
}

int pimc_set_sweep_form(pimc_t h, int form)
{
    if (!h) return PIMC_ERR_ARG;
    if (form != PIMC_FORM_AUTO && form != PIMC_FORM_GENERAL) return fail(h, PIMC_ERR_ARG, "unknown sweep form %d", form);
    h->form = form;
    choose_grid(h);
    return PIMC_OK;
}

int pimc_set_wait_limit(pimc_t h, int64_t ns)
{
    if (!h || ns < 1000) return h ? fail(h, PIMC_ERR_ARG, "wait limit must be >= 1000 ns") : PIMC_ERR_ARG;
    h->wait_ns = ns;
    h->ctx_version++;  // captured into the HMC graph
    return PIMC_OK;
}

int pimc_debug_fix_sum(const double* terms, int64_t n, int as_float, double* out)
{
    if (n < 0 || n > (1 << 20) || (n > 0 && !terms) || !out) {
        set_thread_error("pimc_debug_fix_sum: 0 <= n <= 2^20 terms and an output are required");
        return PIMC_ERR_ARG;
    }
    double* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * (size_t)(n + 1));
    if (e == cudaSuccess && n > 0) e = cudaMemcpy(d, terms, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_fix_sum(d, n, as_float, d + n, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, d + n, sizeof(double), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return PIMC_ERR_CUDA;
    }
    return PIMC_OK;
}

int pimc_debug_map_rate(int packed, int ctas_per_sm, int64_t iters, double* maps_per_s)
{
    if ((ctas_per_sm != 1 && ctas_per_sm != 2 && ctas_per_sm != 4) || iters < 1 || iters > ((int64_t)1 << 24) ||
        !maps_per_s || packed < 0 || packed > 2) {
        set_thread_error("pimc_debug_map_rate: form in {0, 1, 2}, ctas_per_sm in {1, 2, 4}, 1 <= iters <= 2^24 "
                         "and an output required");
        return PIMC_ERR_ARG;
    }
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    float* out = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * (size_t)n_sm * ctas_per_sm * 256);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch_map_rate(packed, ctas_per_sm, n_sm, 16, out, 0);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) e = launch_map_rate(packed, ctas_per_sm, n_sm, iters, out, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return PIMC_ERR_CUDA;
    }
    const double maps = (double)n_sm * ctas_per_sm * 256 * (double)iters * (packed == 1 ? 2.0 : 1.0);
    *maps_per_s = maps / (ms * 1e-3);
    return PIMC_OK;
}

int pimc_debug_lane_maps(const double* X, const double* I_inj, const double* p, double dt, int64_t n, double* f_out,
                         int64_t* n_mismatch)
{
    if (n < 1 || n > (1 << 22) || !X || !I_inj || !p || !f_out || !n_mismatch || !(dt > 0.0)) {
        set_thread_error("pimc_debug_lane_maps: 1 <= n <= 2^22 sites, dt > 0 and all arrays are required");
        return PIMC_ERR_ARG;
    }
    const size_t nx = sizeof(double) * 4 * (size_t)n, ni = sizeof(double) * (size_t)n, np = sizeof(double) * 8;
    char* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * nx + ni + np + 256);
    double* dX = (double*)d;
    double* dF = (double*)(d + nx);
    double* dI = (double*)(d + 2 * nx);
    double* dp = (double*)(d + 2 * nx + ni);
    unsigned* dm = (unsigned*)(d + 2 * nx + ni + np);
    if (e == cudaSuccess) e = cudaMemcpy(dX, X, nx, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dI, I_inj, ni, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dp, p, sizeof(double) * 7, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dm, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = launch_lane_maps(dX, dI, dp, dt, n, dF, dm, 0);
    unsigned m = 0u;
    if (e == cudaSuccess) e = cudaMemcpy(f_out, dF, nx, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&m, dm, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return PIMC_ERR_CUDA;
    }
    *n_mismatch = (int64_t)m;
    return PIMC_OK;
}

int pimc_debug_check_counts(pimc_t h, uint32_t* even, uint32_t* odd, uint32_t* param, uint64_t* moves, int* status,
                            int reset)
{
    if (!h) return PIMC_ERR_ARG;
    if (!checked_build()) return fail(h, PIMC_ERR_STATE, "not a checked build (compile with PIMC_CHECK)");
    CK(h, cudaStreamSynchronize(h->stream));
    const int64_t n1 = h->M + 1;
    uint32_t* outs[3] = {even, odd, param};
    for (int k = 0; k < 3; ++k)
        if (outs[k]) CK(h, cudaMemcpy(outs[k], h->chk + k * h->ldx, sizeof(uint32_t) * n1, cudaMemcpyDeviceToHost));
    if (moves) CK(h, cudaMemcpy(moves, h->chk + 3 * h->ldx, sizeof(uint64_t), cudaMemcpyDeviceToHost));
    int r = pull_state(h);
    if (r != PIMC_OK) return r;
    if (status) *status = h->hs.status;
    if (reset) {
        CK(h, cudaMemsetAsync(h->chk, 0, sizeof(unsigned) * (3 * h->ldx + 2), h->stream));
        h->hs.status &= ~kStatusBounds;
        if ((r = push_state(h)) != PIMC_OK) return r;
    }
    return PIMC_OK;
}

int pimc_debug_skip_arrive(pimc_t h, int cta)
{
    if (!h) return PIMC_ERR_ARG;
    h->skip_cta = cta;
    h->ctx_version++;  // captured into the HMC graph
    return PIMC_OK;
}

int pimc_set_grid(pimc_t h, int grid)
{
    if (h) h->ctx_version++;
    if (!h || grid < 0) return h ? fail(h, PIMC_ERR_ARG, "grid must be >= 0") : PIMC_ERR_ARG;
    h->grid_override = grid;
    choose_grid(h);
    return PIMC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoints: "PIMCCKPT" magic, version, then a payload of fixed-size
// sections, then a CRC-32 (IEEE 802.3 polynomial, reflected) of the payload.
// ---------------------------------------------------------------------------
namespace {

uint32_t crc32(const unsigned char* d, size_t n)
{
    uint32_t c = 0xFFFFFFFFu;
    for (size_t i = 0; i < n; ++i) {
        c ^= d[i];
        for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
    }
    return ~c;
}

struct Writer {
    std::vector<unsigned char> b;
    void put(const void* p, size_t n) { b.insert(b.end(), (const unsigned char*)p, (const unsigned char*)p + n); }
    template <class T> void val(const T& v) { put(&v, sizeof v); }
};

struct Reader {
    const unsigned char* p;
    size_t n, off = 0;
    bool get(void* d, size_t k)
    {
        if (off + k > n) return false;
        memcpy(d, p + off, k);
        off += k;
        return true;
    }
    template <class T> bool val(T& v) { return get(&v, sizeof v); }
};

const char kMagic[8] = {'P', 'I', 'M', 'C', 'C', 'K', 'P', 'T'};
const uint32_t kVersion = 3;

}  // namespace

extern "C" int pimc_checkpoint_save(pimc_t h, const char* path)
{
    if (!h || !path) return h ? fail(h, PIMC_ERR_ARG, "path is NULL") : PIMC_ERR_ARG;
    int r = pull_state(h);
    if (r != PIMC_OK) return r;
    const int64_t n1 = h->M + 1, nd = (int64_t)h->D * n1, nc = nd + h->NP;
    std::vector<double> X(nd), S(nd), F0((size_t)nd), F1((size_t)nd), S1(nc), S2(nc), SH(nc);
    if ((r = get_rows(h, X.data(), h->X, h->ldx, n1)) != PIMC_OK) return r;
    if ((r = get_rows(h, S.data(), h->sig, h->ldx, n1)) != PIMC_OK) return r;
    if ((r = get_rows(h, F0.data(), h->F[0], h->ldf, n1)) != PIMC_OK) return r;
    if ((r = get_rows(h, F1.data(), h->F[1], h->ldf, n1)) != PIMC_OK) return r;
    std::vector<uint32_t> acc((size_t)n1);
    CK(h, cudaMemcpy(acc.data(), h->acc_win, sizeof(uint32_t) * n1, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(S1.data(), h->S1, sizeof(double) * nc, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(S2.data(), h->S2, sizeof(double) * nc, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(SH.data(), h->shift, sizeof(double) * nc, cudaMemcpyDeviceToHost));
    std::vector<unsigned long long> hist;
    std::vector<int64_t> hc(h->n_sel);
    std::vector<double> hl(h->n_sel), hh(h->n_sel);
    if (h->n_sel > 0) {
        hist.resize((size_t)h->n_sel * (h->n_bins + 2));
        CK(h, cudaMemcpy(hist.data(), h->hist, sizeof(unsigned long long) * hist.size(), cudaMemcpyDeviceToHost));
        CK(h, cudaMemcpy(hc.data(), h->h_comp, sizeof(int64_t) * h->n_sel, cudaMemcpyDeviceToHost));
        CK(h, cudaMemcpy(hl.data(), h->h_lo, sizeof(double) * h->n_sel, cudaMemcpyDeviceToHost));
        CK(h, cudaMemcpy(hh.data(), h->h_hi, sizeof(double) * h->n_sel, cudaMemcpyDeviceToHost));
    }
    Writer w;
    w.val(h->model); w.val(h->prec); w.val(h->M); w.val(h->D); w.val(h->NP); w.val(h->scheme); w.val(h->proposal);
    w.val(h->dt); w.val(h->Rm); w.put(h->Rf, sizeof h->Rf);
    w.val(h->n_init); w.val(h->n_skip); w.val(h->n_cool);
    w.val(h->beta0); w.val(h->fbeta); w.val(h->f_acc); w.val(h->alpha); w.val(h->chain);
    w.val(h->hs);
    std::vector<double> yh(n1), Ih(h->M);
    CK(h, cudaMemcpy(yh.data(), h->y64, sizeof(double) * n1, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(Ih.data(), h->I64, sizeof(double) * h->M, cudaMemcpyDeviceToHost));
    w.put(yh.data(), sizeof(double) * n1);
    w.put(Ih.data(), sizeof(double) * h->M);
    w.put(X.data(), sizeof(double) * nd);
    w.put(S.data(), sizeof(double) * nd);
    w.put(F0.data(), sizeof(double) * F0.size());
    w.put(F1.data(), sizeof(double) * F1.size());
    w.put(acc.data(), sizeof(uint32_t) * n1);
    w.put(S1.data(), sizeof(double) * nc);
    w.put(S2.data(), sizeof(double) * nc);
    w.put(SH.data(), sizeof(double) * nc);
    {
        const int64_t nr = (int64_t)(h->D + 1) * h->M;
        std::vector<double> R1(nr), R2(nr);
        CK(h, cudaMemcpy(R1.data(), h->R1, sizeof(double) * nr, cudaMemcpyDeviceToHost));
        CK(h, cudaMemcpy(R2.data(), h->R2, sizeof(double) * nr, cudaMemcpyDeviceToHost));
        w.put(R1.data(), sizeof(double) * nr);
        w.put(R2.data(), sizeof(double) * nr);
    }
    w.val(h->n_sel); w.val(h->n_bins);
    if (h->n_sel > 0) {
        w.put(hc.data(), sizeof(int64_t) * hc.size());
        w.put(hl.data(), sizeof(double) * hl.size());
        w.put(hh.data(), sizeof(double) * hh.size());
        w.put(hist.data(), sizeof(unsigned long long) * hist.size());
    }
    const uint32_t crc = crc32(w.b.data(), w.b.size());
    const uint64_t len = w.b.size();
    FILE* f = fopen(path, "wb");
    if (!f) return fail(h, PIMC_ERR_IO, "cannot open %s for writing", path);
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(&kVersion, 4, 1, f) == 1 && fwrite(&len, 8, 1, f) == 1 &&
              fwrite(w.b.data(), 1, w.b.size(), f) == w.b.size() && fwrite(&crc, 4, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    return ok ? PIMC_OK : fail(h, PIMC_ERR_IO, "short write to %s", path);
}

extern "C" int pimc_checkpoint_load(pimc_t h, const char* path)
{
    if (!h || !path) return h ? fail(h, PIMC_ERR_ARG, "path is NULL") : PIMC_ERR_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(h, PIMC_ERR_IO, "cannot open %s", path);
    char magic[8];
    uint32_t ver = 0, crc = 0;
    uint64_t len = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 && fread(&ver, 4, 1, f) == 1 &&
              ver == kVersion && fread(&len, 8, 1, f) == 1 && len < ((uint64_t)1 << 40);
    std::vector<unsigned char> buf;
    if (ok) {
        buf.resize((size_t)len);
        ok = fread(buf.data(), 1, buf.size(), f) == buf.size() && fread(&crc, 4, 1, f) == 1;
    }
    fclose(f);
    if (!ok) return fail(h, PIMC_ERR_IO, "%s: not a checkpoint of this version, or truncated", path);
    if (crc32(buf.data(), buf.size()) != crc) return fail(h, PIMC_ERR_IO, "%s: CRC mismatch", path);
    Reader rd{buf.data(), buf.size()};
    int model, prec, D, NP, scheme, proposal;
    int64_t M;
    double dt, Rm, Rf[4];
    ok = rd.val(model) && rd.val(prec) && rd.val(M) && rd.val(D) && rd.val(NP) && rd.val(scheme) &&
         rd.val(proposal) && rd.val(dt) && rd.val(Rm) && rd.get(Rf, sizeof Rf);
    if (!ok || model != h->model || M != h->M || D != h->D || NP != h->NP)
        return fail(h, PIMC_ERR_IO, "%s: checkpoint of a different problem shape", path);
    h->dt = dt; h->Rm = Rm;
    h->scheme = scheme; h->proposal = proposal;
    memcpy(h->Rf, Rf, sizeof Rf);
    DevState hs{};
    ok = rd.val(h->n_init) && rd.val(h->n_skip) && rd.val(h->n_cool) && rd.val(h->beta0) && rd.val(h->fbeta) &&
         rd.val(h->f_acc) && rd.val(h->alpha) && rd.val(h->chain) && rd.val(hs);
    const int64_t n1 = M + 1, nd = (int64_t)D * n1, nc = nd + NP;
    std::vector<double> y(n1), I(M), X(nd), S(nd), F0((size_t)nd), F1((size_t)nd), S1(nc), S2(nc), SH(nc);
    std::vector<uint32_t> acc(n1);
    ok = ok && rd.get(y.data(), sizeof(double) * n1) && rd.get(I.data(), sizeof(double) * M) &&
         rd.get(X.data(), sizeof(double) * nd) && rd.get(S.data(), sizeof(double) * nd) &&
         rd.get(F0.data(), sizeof(double) * F0.size()) && rd.get(F1.data(), sizeof(double) * F1.size()) &&
         rd.get(acc.data(), sizeof(uint32_t) * n1) && rd.get(S1.data(), sizeof(double) * nc) &&
         rd.get(S2.data(), sizeof(double) * nc) && rd.get(SH.data(), sizeof(double) * nc);
    const int64_t nr = (int64_t)(D + 1) * M;
    std::vector<double> R1(nr), R2(nr);
    ok = ok && rd.get(R1.data(), sizeof(double) * nr) && rd.get(R2.data(), sizeof(double) * nr);
    int n_sel = 0, n_bins = 0;
    ok = ok && rd.val(n_sel) && rd.val(n_bins);
    if (!ok) return fail(h, PIMC_ERR_IO, "%s: truncated payload", path);
    std::vector<int64_t> hc(n_sel > 0 ? n_sel : 0);
    std::vector<double> hl(hc.size()), hh(hc.size());
    std::vector<unsigned long long> hist;
    if (n_sel > 0) {
        hist.resize((size_t)n_sel * (n_bins + 2));
        ok = rd.get(hc.data(), sizeof(int64_t) * n_sel) && rd.get(hl.data(), sizeof(double) * n_sel) &&
             rd.get(hh.data(), sizeof(double) * n_sel) &&
             rd.get(hist.data(), sizeof(unsigned long long) * hist.size());
        if (!ok) return fail(h, PIMC_ERR_IO, "%s: truncated histogram section", path);
    }
    CK(h, cudaStreamSynchronize(h->stream));
    h->prec = prec;
    int r = upload_data(h, y.data(), I.data());
    if (r != PIMC_OK) return r;
    CK(h, cudaStreamSynchronize(h->stream));
    h->have_data = true;
    h->have_params = true;
    if ((r = put_rows(h, h->X, X.data())) != PIMC_OK) return r;
    if ((r = put_rows(h, h->sig, S.data())) != PIMC_OK) return r;
    // cache rows are [D][M+1] with stride ldf
    {
        const size_t es = esize(h);
        std::vector<unsigned char> t((size_t)D * n1 * es);
        for (int b = 0; b < 2; ++b) {
            const std::vector<double>& src = b == 0 ? F0 : F1;
            for (size_t i = 0; i < src.size(); ++i) {
                if (prec == PIMC_FP64) memcpy(&t[i * es], &src[i], es);
                else { float v = (float)src[i]; memcpy(&t[i * es], &v, es); }
            }
            CK(h, cudaMemcpy2DAsync(h->F[b], es * h->ldf, t.data(), es * n1, es * n1, D, cudaMemcpyHostToDevice,
                                    h->stream));
            CK(h, cudaStreamSynchronize(h->stream));  // t is refilled for the other buffer
        }
    }
    // on the handle's stream, complete before the host arrays go
    CK(h, cudaMemcpyAsync(h->acc_win, acc.data(), sizeof(uint32_t) * n1, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->S1, S1.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->S2, S2.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->shift, SH.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->R1, R1.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->R2, R2.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, h->stream));
    if (n_sel > 0) {
        if ((r = pimc_set_histograms(h, n_sel, hc.data(), hl.data(), hh.data(), n_bins)) != PIMC_OK) return r;
        CK(h, cudaMemcpyAsync(h->hist, hist.data(), sizeof(unsigned long long) * hist.size(), cudaMemcpyHostToDevice,
                              h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    hs.status = 0;
    hs.abort = 0;
    h->hs = hs;
    h->ctx_version++;
    CK(h, cudaMemsetAsync(h->bar, 0, sizeof(unsigned) * 4, h->stream));
    choose_grid(h);
    return push_state(h);
}

// ---------------------------------------------------------------------------
// Batched launch of many chains (independent data sets and/or chains).
// ---------------------------------------------------------------------------
struct pimc_batch_s {
    std::vector<pimc_t> hs;
    int model = 0, prec = 0;
    cudaStream_t stream = nullptr;
    Ctx* d_ctx = nullptr;
    int* d_first = nullptr;
    BatchItem* d_items = nullptr;
    int n_ctas = 0, nt = 256, ctas_per_sm = 0;
    int split = 1;          // most CTAs one chain may be split over
    int n_split = 0;        // chains split over several CTAs in the current plan
    std::vector<unsigned> versions;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_sweeps = -1;
    uint64_t graph_seed = 0;
    bool dirty = true;
    std::string err;
};

namespace {

int bfail(pimc_batch_t b, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_create_error = buf;
    return code;
}

#define BCK(b, call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? PIMC_ERR_OOM : PIMC_ERR_CUDA, \
                         "%s: %s", #call, cudaGetErrorString(e_));                            \
    } while (0)

// Work of one sweep of a chain: sites x (1 + free parameters).
double chain_cost(pimc_t h)
{
    int nf = 0;
    for (int l = 0; l < h->NP; ++l) nf += (h->hs.free_mask >> l) & 1u;
    return (double)(h->M + 1) * (double)(1 + nf);
}

// Contexts of all chains and their assignment to CTAs, longest first.  With
// split > 1, a chain costing more than the mean load of a CTA is cut into up
// to `split` tiles (at least 2 nt sites each), which go to that many of the
// currently least loaded CTAs; every other chain goes whole to the least
// loaded CTA.  Each CTA's items are appended in one global order (decreasing
// cost), so the CTAs sharing a split chain always reach it without a cycle of
// waits.
int batch_build(pimc_batch_t b)
{
    const int n = (int)b->hs.size();
    const int sms = b->hs[0]->num_sms;
    int occ = batch_ctas_per_sm(b->model, b->prec, b->nt);
    if (occ < 1) return bfail(b, PIMC_ERR_CUDA, "batched kernel cannot be resident (nt = %d)", b->nt);
    int per_sm = b->ctas_per_sm > 0 ? std::min(b->ctas_per_sm, occ) : occ;
    std::vector<double> cost(n);
    double total = 0.0;
    for (int i = 0; i < n; ++i) total += (cost[i] = chain_cost(b->hs[i]));
    // enough CTAs for every chain, or for every tile when chains are split
    b->n_ctas = std::max(1, std::min(b->split > 1 ? per_sm * sms : n, per_sm * sms));
    std::vector<Ctx> ctx(n);
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) {
        ctx[i] = make_ctx(b->hs[i]);
        idx[i] = i;
        b->versions[i] = b->hs[i]->ctx_version;
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    const double target = total / b->n_ctas;
    std::vector<double> load(b->n_ctas, 0.0);
    std::vector<std::vector<BatchItem>> per(b->n_ctas);
    std::vector<int> by_load(b->n_ctas);
    b->n_split = 0;
    for (int i : idx) {
        int g = 1;
        if (b->split > 1 && cost[i] > target) {
            const int64_t max_tiles = std::max<int64_t>(1, (b->hs[i]->M + 1) / (2 * b->nt));
            g = (int)std::min<int64_t>({(int64_t)b->split, (int64_t)std::ceil(cost[i] / target), max_tiles,
                                        (int64_t)b->n_ctas});
            g = std::max(g, 1);
        }
        for (int k = 0; k < b->n_ctas; ++k) by_load[k] = k;
        std::partial_sort(by_load.begin(), by_load.begin() + g, by_load.end(),
                          [&](int a, int c) { return load[a] < load[c] || (load[a] == load[c] && a < c); });
        std::sort(by_load.begin(), by_load.begin() + g);
        for (int r = 0; r < g; ++r) {
            per[by_load[r]].push_back(BatchItem{i, r, g, 0});
            load[by_load[r]] += cost[i] / g;
        }
        if (g > 1) b->n_split++;
    }
    std::vector<int> first(b->n_ctas + 1, 0);
    std::vector<BatchItem> items;
    items.reserve(n + 64);
    for (int k = 0; k < b->n_ctas; ++k) {
        first[k] = (int)items.size();
        for (const BatchItem& it : per[k]) items.push_back(it);
    }
    first[b->n_ctas] = (int)items.size();
    if (b->d_ctx) cudaFree(b->d_ctx);
    if (b->d_first) cudaFree(b->d_first);
    if (b->d_items) cudaFree(b->d_items);
    b->d_ctx = nullptr; b->d_first = nullptr; b->d_items = nullptr;
    BCK(b, cudaMalloc(&b->d_ctx, sizeof(Ctx) * n));
    BCK(b, cudaMalloc(&b->d_first, sizeof(int) * (b->n_ctas + 1)));
    BCK(b, cudaMalloc(&b->d_items, sizeof(BatchItem) * items.size()));
    // on the batch's stream (its launches follow), complete before the host vectors go
    BCK(b, cudaMemcpyAsync(b->d_ctx, ctx.data(), sizeof(Ctx) * n, cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaMemcpyAsync(b->d_first, first.data(), sizeof(int) * (b->n_ctas + 1), cudaMemcpyHostToDevice,
                           b->stream));
    BCK(b, cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                           b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->dirty = false;
    return PIMC_OK;
}

cudaError_t batch_launch(pimc_batch_t b, int64_t n_sweeps, uint64_t seed)
{
    return launch_batch_sweep(b->model, b->prec, b->nt, b->d_ctx, b->d_first, b->d_items, b->n_ctas, n_sweeps, seed,
                              b->n_split > 0, b->stream);
}

struct Tuning {
    int nt, ctas_per_sm, split;
};
std::map<std::pair<int, int>, Tuning>& tune_cache()
{
    static std::map<std::pair<int, int>, Tuning> m;
    return m;
}

int tune_key_sites(pimc_batch_t b)
{
    double tot = 0.0;
    for (pimc_t h : b->hs) tot += chain_cost(h);
    return (int)std::log2(std::max(1.0, tot)) * 16 + b->model * 4 + b->prec;
}

}  // namespace

extern "C" {

int pimc_batch_create(pimc_batch_t* out, const pimc_t* handles, int n)
{
    if (!out || !handles || n < 1) return bfail(nullptr, PIMC_ERR_ARG, "bad batch arguments");
    *out = nullptr;
    pimc_batch_t b = new pimc_batch_s();
    for (int i = 0; i < n; ++i) {
        pimc_t h = handles[i];
        if (!h) { delete b; return bfail(nullptr, PIMC_ERR_ARG, "handle %d is NULL", i); }
        if (!h->have_data || !h->have_params) { delete b; return bfail(nullptr, PIMC_ERR_STATE, "handle %d has no data/params", i); }
        if (i > 0 && (h->model != handles[0]->model || h->prec != handles[0]->prec || h->device != handles[0]->device)) {
            delete b;
            return bfail(nullptr, PIMC_ERR_ARG, "handles of a batch must share model, precision and device");
        }
        if (cudaStreamSynchronize(h->stream) != cudaSuccess || pull_state(h) != PIMC_OK) {
            delete b;
            return bfail(nullptr, PIMC_ERR_CUDA, "handle %d: synchronisation failed", i);
        }
        b->hs.push_back(h);
    }
    b->model = handles[0]->model;
    b->prec = handles[0]->prec;
    b->stream = handles[0]->stream;
    b->versions.assign(n, ~0u);
    auto it = tune_cache().find(std::make_pair(tune_key_sites(b), n));
    if (it != tune_cache().end()) {
        b->nt = it->second.nt;
        b->ctas_per_sm = it->second.ctas_per_sm;
        b->split = it->second.split;
    }
    int r = batch_build(b);
    if (r != PIMC_OK) {
        g_create_error = b->err;
        pimc_batch_destroy(b);
        return r;
    }
    *out = b;
    return PIMC_OK;
}

int pimc_batch_destroy(pimc_batch_t b)
{
    if (!b) return PIMC_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->d_ctx) cudaFree(b->d_ctx);
    if (b->d_first) cudaFree(b->d_first);
    if (b->d_items) cudaFree(b->d_items);
    delete b;
    return PIMC_OK;
}

const char* pimc_batch_last_error(pimc_batch_t b) { return b ? b->err.c_str() : g_create_error.c_str(); }

int pimc_batch_set_tuning(pimc_batch_t b, int threads_per_cta, int ctas_per_sm, int ctas_per_chain)
{
    if (!b) return PIMC_ERR_ARG;
    if (threads_per_cta != 128 && threads_per_cta != 256) return bfail(b, PIMC_ERR_ARG, "threads_per_cta must be 128 or 256");
    if (ctas_per_sm < 0) return bfail(b, PIMC_ERR_ARG, "ctas_per_sm must be >= 0");
    if (ctas_per_chain < 1 || ctas_per_chain > 64) return bfail(b, PIMC_ERR_ARG, "ctas_per_chain must be in [1, 64]");
    BCK(b, cudaStreamSynchronize(b->stream));
    b->nt = threads_per_cta;
    b->ctas_per_sm = ctas_per_sm;
    b->split = ctas_per_chain;
    return batch_build(b);
}

int pimc_batch_info(pimc_batch_t b, int* n_ctas, int* threads_per_cta, int* n_split)
{
    if (!b) return PIMC_ERR_ARG;
    if (n_ctas) *n_ctas = b->n_ctas;
    if (threads_per_cta) *threads_per_cta = b->nt;
    if (n_split) *n_split = b->n_split;
    return PIMC_OK;
}

int pimc_batch_sweep(pimc_batch_t b, int64_t n_sweeps, uint64_t seed)
{
    if (!b) return PIMC_ERR_ARG;
    if (n_sweeps < 0) return bfail(b, PIMC_ERR_ARG, "n_sweeps < 0");
    for (size_t i = 0; i < b->hs.size(); ++i)
        if (b->hs[i]->ctx_version != b->versions[i]) b->dirty = true;
    if (b->dirty) {
        BCK(b, cudaStreamSynchronize(b->stream));
        int r = batch_build(b);
        if (r != PIMC_OK) return r;
    }
    if (n_sweeps == 0) return PIMC_OK;
    // a sweep block is a sequence of launches of <= 256 sweeps each (bounded
    // kernel duration), captured once as a CUDA graph and replayed
    const int64_t chunk = 256;
    if (!b->exec || b->graph_sweeps != n_sweeps || b->graph_seed != seed) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        if (b->stream) {
            cudaGraph_t graph = nullptr;
            BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int64_t done = 0; done < n_sweeps && e == cudaSuccess; done += chunk)
                e = batch_launch(b, std::min<int64_t>(chunk, n_sweeps - done), seed);
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            BCK(b, e);
            b->graph_sweeps = n_sweeps;
            b->graph_seed = seed;
        }
    }
    if (b->exec) {
        BCK(b, cudaGraphLaunch(b->exec, b->stream));
    } else {
        for (int64_t done = 0; done < n_sweeps; done += chunk)
            BCK(b, batch_launch(b, std::min<int64_t>(chunk, n_sweeps - done), seed));
    }
    return PIMC_OK;
}

int pimc_batch_sync(pimc_batch_t b)
{
    if (!b) return PIMC_ERR_ARG;
    BCK(b, cudaStreamSynchronize(b->stream));
    return PIMC_OK;
}

int pimc_batch_autotune(pimc_batch_t b, int64_t trial_sweeps, uint64_t seed, int* threads_per_cta, int* ctas_per_sm,
                        int* ctas_per_chain)
{
    if (!b) return PIMC_ERR_ARG;
    if (trial_sweeps < 1) return bfail(b, PIMC_ERR_ARG, "trial_sweeps must be >= 1");
    BCK(b, cudaStreamSynchronize(b->stream));
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    float best = 1e30f;
    Tuning best_t{b->nt, b->ctas_per_sm, b->split};
    const int nts[2] = {128, 256};
    const int splits[3] = {1, 2, 4};
    for (int ni = 0; ni < 2; ++ni) {
        const int occ = batch_ctas_per_sm(b->model, b->prec, nts[ni]);
        for (int k = 1; k <= occ; k *= 2) {
            for (int si = 0; si < 3; ++si) {
                b->nt = nts[ni];
                b->ctas_per_sm = k;
                b->split = splits[si];
                int r = batch_build(b);
                if (r != PIMC_OK) return r;
                if (splits[si] > 1 && b->n_split == 0) continue;  // nothing to split: same as split 1
                BCK(b, cudaEventRecord(e0, b->stream));
                BCK(b, batch_launch(b, trial_sweeps, seed));
                BCK(b, cudaEventRecord(e1, b->stream));
                BCK(b, cudaEventSynchronize(e1));
                float ms = 0.0f;
                BCK(b, cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    best_t = Tuning{nts[ni], k, splits[si]};
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->nt = best_t.nt;
    b->ctas_per_sm = best_t.ctas_per_sm;
    b->split = best_t.split;
    tune_cache()[std::make_pair(tune_key_sites(b), (int)b->hs.size())] = best_t;
    if (threads_per_cta) *threads_per_cta = best_t.nt;
    if (ctas_per_sm) *ctas_per_sm = best_t.ctas_per_sm;
    if (ctas_per_chain) *ctas_per_chain = best_t.split;
    return batch_build(b);
}

}  // extern "C"
