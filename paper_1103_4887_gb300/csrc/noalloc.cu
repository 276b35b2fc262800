// Allocation-free variant of the global-action kernel.
//
// Some callers cannot allocate device memory at call time: code running
// under a fixed memory budget or a caller-owned memory pool, plugin hosts that
// forbid cudaMalloc/cudaFree on their threads, and real-time loops where an
// allocation (which may synchronise the device) is not allowed.  For them,
// pimc_action_static computes the FP64 action of the explicit RK4 model error
// (what pimc_action_dev gives for an FP64 handle with the RK4 scheme and model
// HH, LINGAUSS or TOY1D) without a handle and without allocating: its per-CTA partial sums and its
// last-block counter live in one file-scope __device__ array, held by every
// GPU that loads this library until the process exits.
#include <cstdio>

#include "../../include/pimc.h"
#include "device.cuh"
#include "internal.h"

namespace pimc {
namespace {

constexpr int kStaticBlock = 128;
constexpr int kStaticMaxCtas = 2048;                 // one CTA per 128 sites
constexpr int64_t kStaticMaxM = (int64_t)kStaticMaxCtas * kStaticBlock - 1;
constexpr size_t kCounterBytes = 256;                // [0, 256): last-block counter
constexpr size_t kScratchBytes = kCounterBytes + sizeof(double) * 2 * kStaticMaxCtas;  // 33,024 bytes

// The shared scratch: counter, then 2 doubles (A_o, A_f) per CTA.
static __device__ __align__(256) unsigned char g_action_scratch[kScratchBytes];

template <class Model>
__global__ void __launch_bounds__(kStaticBlock)
action_static_kernel(int64_t M, double dt, double Rm, double Rf0, double Rf1, double Rf2, double Rf3,
                     const double* X, const double* p, const double* y, const double* I, double* out,
                     unsigned char* scratch)
{
    constexpr int D = Model::D;
    __shared__ double wsum[2][kStaticBlock / 32];
    __shared__ int last;
    unsigned* counter = (unsigned*)scratch;
    double* part = (double*)(scratch + kCounterBytes);
    const double Rf[4] = {Rf0, Rf1, Rf2, Rf3};
    double q[kMaxP];
    Model::prep(p, q);
    double v[2] = {0.0, 0.0};
    const int64_t n = (int64_t)blockIdx.x * kStaticBlock + threadIdx.x;
    if (n <= M) {
        double x[D];
        for (int a = 0; a < D; ++a) x[a] = X[a * (M + 1) + n];
        if (n >= 1) {
            const double d = x[0] - y[n];
            v[0] = 0.5 * Rm * d * d;
        }
        if (n < M) {
            double f[D];
            rk4_map<Model, double>(x, q, I[n], dt, f);
            for (int a = 0; a < D; ++a) {
                const double e = X[a * (M + 1) + n + 1] - f[a];
                v[1] += 0.5 * Rf[a] * e * e;
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 2; ++k) {
        double w = v[k];
        for (int off = 16; off > 0; off >>= 1) w += __shfl_down_sync(0xffffffffu, w, off);
        if (lane == 0) wsum[k][wid] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 2; ++k) {
            double t = 0.0;
            for (int j = 0; j < kStaticBlock / 32; ++j) t += wsum[k][j];
            part[2 * blockIdx.x + k] = t;
        }
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t[2] = {0.0, 0.0};
        for (unsigned i = 0; i < gridDim.x; ++i)
            for (int k = 0; k < 2; ++k) t[k] += __ldcg(&part[2 * i + k]);
        out[0] = t[0] + t[1];
        out[1] = t[0];
        out[2] = t[1];
        *counter = 0u;
    }
}

// Device address of the scratch array in the current device's context.  It is
// looked up on every call (cudaGetSymbolAddress allocates nothing and costs a
// table lookup): an address cached from an earlier call would belong to a
// context that no longer exists after cudaDeviceReset, or that is not current
// when the caller has made another context current.
int scratch_address(void** ptr)
{
    void* a = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&a, g_action_scratch);
    if (e != cudaSuccess || !a) {
        char msg[160];
        snprintf(msg, sizeof msg, "pimc_action_static: cudaGetSymbolAddress of the scratch array failed: %s",
                 cudaGetErrorString(e));
        set_thread_error(msg);
        return PIMC_ERR_CUDA;
    }
    *ptr = a;
    return PIMC_OK;
}

}  // namespace
}  // namespace pimc

extern "C" int pimc_action_static(int model, int64_t M, double dt, double Rm, const double* Rf,
                                  const double* X_dev, const double* p_dev, const double* y_dev,
                                  const double* I_dev, double* out_dev, void* stream)
{
    using namespace pimc;
    int D;
    switch (model) {
    case PIMC_MODEL_HH: D = 4; break;
    case PIMC_MODEL_LINGAUSS: D = 2; break;
    case PIMC_MODEL_TOY1D: D = 1; break;
    case PIMC_MODEL_HH_PAPER:
        set_thread_error("pimc_action_static: PIMC_MODEL_HH_PAPER is not supported by this entry point "
                         "(models HH, LINGAUSS and TOY1D with the RK4 model error only)");
        return PIMC_ERR_ARG;
    default: set_thread_error("pimc_action_static: unknown model"); return PIMC_ERR_ARG;
    }
    if (M < 1 || M > kStaticMaxM) {
        char msg[160];
        snprintf(msg, sizeof msg, "pimc_action_static: M = %lld outside [1, %lld], the capacity of its fixed scratch",
                 (long long)M, (long long)kStaticMaxM);
        set_thread_error(msg);
        return PIMC_ERR_ARG;
    }
    if (!(dt > 0.0) || !(Rm > 0.0) || !Rf || !X_dev || !p_dev || !y_dev || !I_dev || !out_dev) {
        set_thread_error("pimc_action_static: bad dt/Rm or NULL pointer");
        return PIMC_ERR_ARG;
    }
    double rf[4] = {0.0, 0.0, 0.0, 0.0};
    for (int a = 0; a < D; ++a) rf[a] = Rf[a];
    void* scratch = nullptr;
    int r = scratch_address(&scratch);
    if (r != PIMC_OK) return r;
    cudaStream_t s = (cudaStream_t)stream;
    // the counter must start at zero even if an earlier launch was cut short
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned), s) != cudaSuccess) {
        set_thread_error("pimc_action_static: clearing the scratch counter failed");
        return PIMC_ERR_CUDA;
    }
    const unsigned grid = (unsigned)((M + 1 + kStaticBlock - 1) / kStaticBlock);
    unsigned char* sp = (unsigned char*)scratch;
    if (model == PIMC_MODEL_HH)
        action_static_kernel<HH<double>><<<grid, kStaticBlock, 0, s>>>(M, dt, Rm, rf[0], rf[1], rf[2], rf[3], X_dev,
                                                                      p_dev, y_dev, I_dev, out_dev, sp);
    else if (model == PIMC_MODEL_LINGAUSS)
        action_static_kernel<LinGauss<double>><<<grid, kStaticBlock, 0, s>>>(M, dt, Rm, rf[0], rf[1], rf[2], rf[3],
                                                                            X_dev, p_dev, y_dev, I_dev, out_dev, sp);
    else
        action_static_kernel<Toy1D<double>><<<grid, kStaticBlock, 0, s>>>(M, dt, Rm, rf[0], rf[1], rf[2], rf[3],
                                                                         X_dev, p_dev, y_dev, I_dev, out_dev, sp);
    if (cudaGetLastError() != cudaSuccess) {
        set_thread_error("pimc_action_static: kernel launch failed");
        return PIMC_ERR_CUDA;
    }
    return PIMC_OK;
}
