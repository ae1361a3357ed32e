// Per-shot waveform misfit that allocates no memory.
//
// Some callers cannot allocate device memory when they call into this
// library: an application that hands the GPU's memory to its own pool or
// arena at start-up and forbids any later cudaMalloc, or a runtime that must
// not risk an allocation failure (or the device-wide synchronisation a
// cudaFree implies) in the middle of its time-critical loop.  For them this
// file offers gbfwi_misfit_noalloc: the same residual reduction the misfit
// of gbfwi_adjoint_gradient performs, but with its per-block partial sums in
// a fixed, file-scope device array instead of a library work buffer.
//
// The array is sized for at most GBFWI_NOALLOC_MAX_SHOTS shots and exists on
// every GPU that loads the library's device code until the process exits
// (about 130 KB).  With CUDA's default lazy module loading that device code,
// and with it the array, is loaded on a device by the first call there (the
// symbol lookup below); that first call is the one that can reserve memory,
// so a caller whose pool takes the GPU's memory later makes it before that,
// or sets CUDA_MODULE_LOADING=EAGER so the load happens with the library's.
// All calls share the array and it keeps the contents of the last call:
// calls whose work overlaps on the GPU (different streams, or threads) race
// on it.

#include <cmath>
#include <mutex>

#include "gbfwi_internal.h"

namespace {

constexpr int kMaxShots = GBFWI_NOALLOC_MAX_SHOTS;
constexpr int kBlocksPerShot = 64;
constexpr int kThreads = 256;

// [shot][block] partial sums, then [shot] results, then one flag word
constexpr int kScratchDoubles = kMaxShots * kBlocksPerShot + kMaxShots + 2;
static __device__ __align__(256) double g_misfit_scratch[kScratchDoubles];

// device address of g_misfit_scratch per device ordinal (host code must not
// use the symbol's host-side stand-in as a device pointer)
std::mutex g_mu;
double *g_addr[64];

__global__ void misfit_partials_noalloc(const float *__restrict__ syn, const float *__restrict__ obs,
                                        long long per_shot, double *__restrict__ scratch)
{
    const int shot = blockIdx.y;
    const float *s = syn + (long long)shot * per_shot;
    const float *d = obs + (long long)shot * per_shot;
    double acc = 0.0;
    int bad = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < per_shot;
         q += (long long)gridDim.x * blockDim.x) {
        float r = s[q] - d[q];
        if (!isfinite(r)) bad = 1;
        acc += (double)r * (double)r;
    }
    __shared__ double red[kThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[shot * kBlocksPerShot + blockIdx.x] = red[0];
    if (bad) atomicOr(reinterpret_cast<int *>(scratch + kMaxShots * kBlocksPerShot + kMaxShots), 1);
}

__global__ void misfit_finish_noalloc(double *__restrict__ scratch, int nshot, double half_dt)
{
    int shot = blockIdx.x * blockDim.x + threadIdx.x;
    if (shot >= nshot) return;
    double s = 0.0;
    for (int b = 0; b < kBlocksPerShot; ++b) s += scratch[shot * kBlocksPerShot + b];
    scratch[kMaxShots * kBlocksPerShot + shot] = half_dt * s;
}

// Device address of the scratch array on the current device, looked up once
// per device.
int scratch_on_current_device(double **out)
{
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return GBFWI_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        GB_CUDA(cudaGetSymbolAddress(&p, g_misfit_scratch));
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return GBFWI_OK;
}

}  // namespace

extern "C" int gbfwi_misfit_noalloc(const float *syn, const float *obs, int nshot, long long samples_per_shot,
                                    double dt, double *misfit, void *stream)
{
    if (!syn || !obs || !misfit || nshot < 1 || samples_per_shot < 1 || !(dt > 0)) return GBFWI_EINVAL;
    if (nshot > kMaxShots) return GBFWI_ESCRATCH;
    // syn and obs must be memory of the current device (gb_is_device_ptr
    // rejects another GPU's memory), misfit host memory
    if (!gb_is_device_ptr(syn) || !gb_is_device_ptr(obs) || gb_is_device_ptr(misfit)) return GBFWI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // the call ends with a copy into host stack memory and a stream
    // synchronisation, neither of which a capturing stream accepts
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    GB_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return GBFWI_EINVAL;
    double *scratch = nullptr;
    GB_TRY(scratch_on_current_device(&scratch));
    double *flag = scratch + kMaxShots * kBlocksPerShot + kMaxShots;
    GB_CUDA(cudaMemsetAsync(flag, 0, sizeof(double), s));   // the only state that must start at zero
    misfit_partials_noalloc<<<dim3(kBlocksPerShot, nshot), kThreads, 0, s>>>(syn, obs, samples_per_shot, scratch);
    GB_LAUNCHED();
    misfit_finish_noalloc<<<(nshot + 127) / 128, 128, 0, s>>>(scratch, nshot, 0.5 * dt);
    GB_LAUNCHED();
    // results land in host stack memory first, so that the caller's array is
    // written only on success
    double res[kMaxShots];
    int flag_h = 0;
    GB_CUDA(cudaMemcpyAsync(&flag_h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaMemcpyAsync(res, scratch + kMaxShots * kBlocksPerShot, nshot * sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    GB_CUDA(cudaStreamSynchronize(s));
    if (flag_h != 0) return gb_nonfinite("misfit");
    for (int i = 0; i < nshot; ++i) misfit[i] = res[i];
    return GBFWI_OK;
}
