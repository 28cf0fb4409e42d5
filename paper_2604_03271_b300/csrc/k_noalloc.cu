// k_noalloc.cu -- a tempering step that allocates no memory at all.
//
// Some callers cannot call cudaMalloc: code running inside a host framework
// that owns every device allocation (a fixed arena, a memory pool with a hard
// cap), or a caller that must not let device memory grow once it has started
// serving.  smc_k_reweight_static gives them the reweighting kernel without
// any allocation: the caller passes its device input and output arrays, and
// the kernel's scratch (the job descriptor and the FP64 weight buffer) lives
// in a fixed file-scope device array that every GPU loading this library
// holds until the process exits.
//
// Every call made outside a stream capture looks up the array's device
// address with cudaGetSymbolAddress (with the call's device current), so the
// address stays right after a device reset re-creates the context; a call
// made while its stream is capturing reuses the address found by the last
// uncaptured call on that device, so make one call on each device before any
// capture.  All calls share the one array and it keeps the last call's
// contents; each call rewrites every scratch field it reads.  Calls whose
// kernels overlap on the GPU race on the array.
#include <mutex>

#include "../../include/smc_kernels.h"
#include "kernels.h"

namespace smc {

constexpr int STATIC_MAX_DEVICES = 64;

struct StaticScratch {
    JobDev job;
    int slot;
    int pad_[63];
    double w64[SMC_STATIC_MAX_PARTICLES];
    double rwpart[RW_SPLIT_MAX];  // one partial sum per weights CTA (no components)
};

static __device__ __align__(256) StaticScratch g_scratch;

static std::mutex g_mu;
static StaticScratch *g_addr[STATIC_MAX_DEVICES];

// device address of g_scratch on the current device: looked up again on every
// call outside a stream capture (a device reset gives the array a new
// address), the last address found on this device inside one
static cudaError_t scratch_address(int dev, cudaStream_t s, StaticScratch **out)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (StaticScratch *)p;
    } else if (!g_addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

static int status_of(cudaError_t e)
{
    return e == cudaSuccess ? SMC_OK : (e == cudaErrorMemoryAllocation ? SMC_ENOMEM : SMC_ECUDA);
}

}  // namespace smc

using namespace smc;

extern "C" int smc_k_reweight_static(const void *E_dev, int64_t T, double beta, double rho,
                                     int32_t precision, uint64_t *q_dev, double *delta,
                                     double *logz_inc, int32_t *final_step, void *cuda_stream)
{
    if (!E_dev || !q_dev || !delta || !logz_inc || !final_step) return SMC_EINVAL;
    if (T < 2 || T > SMC_STATIC_MAX_PARTICLES) return SMC_EINVAL;  // beyond the fixed scratch
    if (!(beta >= 0.0 && beta < 1.0) || !(rho > 0.0 && rho < 1.0)) return SMC_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= STATIC_MAX_DEVICES) return SMC_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    StaticScratch *sc = nullptr;
    if (scratch_address(dev, s, &sc) != cudaSuccess) return SMC_ECUDA;

    // a fresh descriptor every call: zero-dimensional job, weights in scratch
    JobDev jb{};
    jb.T = jb.S = (int)T;
    jb.fp64 = precision ? 1 : 0;
    if (precision)
        jb.E64 = (double *)E_dev;
    else
        jb.E = (float *)E_dev;
    jb.w64 = sc->w64;
    jb.rwpart = sc->rwpart;
    jb.q = (unsigned long long *)q_dev;
    jb.d = 0;
    jb.beta = beta;
    jb.rho = rho;
    jb.logz = 0.0;
    jb.state = JOB_ACTIVE;
    jb.max_stages = 1 << 30;
    const int zero = 0;
    cudaError_t e = cudaMemcpyAsync(&sc->job, &jb, sizeof(JobDev), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sc->slot, &zero, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_reweight(&sc->job, &sc->slot, 1, precision != 0, T, s);
    JobDev o{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&o, &sc->job, sizeof(JobDev), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return status_of(e);
    if (o.status != 0) return o.status;
    *delta = o.delta;
    *logz_inc = o.logz;
    *final_step = o.final_step;
    return SMC_OK;
}
