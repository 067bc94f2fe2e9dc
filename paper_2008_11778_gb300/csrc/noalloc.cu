// noalloc.cu -- the misfit reduction without any device allocation.
//
// Some callers cannot allocate device memory while they run: a host
// framework that owns the whole device-memory budget through its own pool or
// caching allocator, or a latency-bound loop that must not pay the implicit
// device-wide synchronisation of cudaMalloc / cudaFree.  For them,
// aafwi_misfit_noalloc computes the same residual and misfit as aafwi_misfit
// but keeps its scratch (the per-chunk FP64 partial sums and the result) in a
// file-scope __device__ array that is part of the loaded library image: every
// GPU that loads the library holds it (512 KB) until the process exits.
//
// The partial sums are taken over fixed chunks of CHUNK samples, one CTA per
// chunk, so the result does not depend on scheduling; the array holds at most
// MAX_CHUNKS partials, which bounds a call to MAX_CHUNKS * CHUNK samples.
#include <string>

#include "../../include/aafwi.h"
#include "internal.cuh"

namespace aafwi {
namespace {

constexpr long long CHUNK = 1LL << 16;
constexpr int MAX_CHUNKS = 1 << 16;
static_assert(CHUNK * MAX_CHUNKS == AAFWI_MISFIT_NOALLOC_MAX_SAMPLES, "header limit");
constexpr int NT = 256;

// partials [0, MAX_CHUNKS) and the misfit J at [MAX_CHUNKS].
static __device__ __align__(256) double g_misfit_scratch[MAX_CHUNKS + 1];

__device__ __forceinline__ double block_sum256(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = threadIdx.x < NT / 32 ? sh[threadIdx.x] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// CTA b reduces chunk b: r = d - o over [b*CHUNK, min((b+1)*CHUNK, n)).
__global__ void __launch_bounds__(NT) k_misfit_chunks(const float *d, const float *o, float *r, long long n,
                                                      double *partials)
{
    __shared__ double sh[NT / 32];
    const long long lo = blockIdx.x * CHUNK;
    const long long hi = lo + CHUNK < n ? lo + CHUNK : n;
    double acc = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += NT) {
        const float e = d[i] - o[i];
        if (r) r[i] = e;
        acc += (double)e * e;
    }
    acc = block_sum256(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// J = 1/2 sum of the nch partials, written to out[0] and, if given, to J_out.
__global__ void __launch_bounds__(NT) k_misfit_finish(const double *partials, int nch, double *out,
                                                      double *J_out)
{
    __shared__ double sh[NT / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nch; i += NT) acc += partials[i];
    acc = block_sum256(acc, sh);
    if (threadIdx.x == 0) {
        out[0] = 0.5 * acc;
        if (J_out) *J_out = 0.5 * acc;
    }
}

// Device address of the scratch array on the current device.  Host code may
// not take the address of a __device__ symbol, so it is looked up on every
// call: the lookup is a host-side query, and a cached address could go stale
// if the device's context were reset and the module loaded again.
cudaError_t scratch_for_current_device(double **out)
{
    double *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_misfit_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace
}  // namespace aafwi

extern "C" {

int aafwi_misfit_noalloc(const float *d_syn, const float *d_obs, long long n, float *resid,
                         double *J_dev, double *J_host, aafwi_stream stream)
{
    using namespace aafwi;
    if (!d_syn || !d_obs || (!J_dev && !J_host)) {
        set_call_error("NULL argument (d_syn, d_obs, and J_dev or J_host are required)");
        return AAFWI_ERR_ARG;
    }
    if (n < 1 || n > CHUNK * MAX_CHUNKS) {
        set_call_error("sample count " + std::to_string(n) + " outside [1, " +
                       std::to_string(CHUNK * MAX_CHUNKS) + "]: the static scratch holds " +
                       std::to_string(MAX_CHUNKS) + " partial sums of " + std::to_string(CHUNK) +
                       " samples");
        return AAFWI_ERR_ARG;
    }
    double *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) {
        set_call_error(std::string("scratch address: ") + cudaGetErrorString(e));
        return AAFWI_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nch = (int)((n + CHUNK - 1) / CHUNK);
    count_launch(2);
    k_misfit_chunks<<<nch, NT, 0, st>>>(d_syn, d_obs, resid, n, scratch);
    k_misfit_finish<<<1, NT, 0, st>>>(scratch, nch, scratch + MAX_CHUNKS, J_dev);
    e = cudaGetLastError();
    if (e == cudaSuccess && J_host) {
        e = cudaMemcpyAsync(J_host, scratch + MAX_CHUNKS, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
        set_call_error(std::string("misfit_noalloc: ") + cudaGetErrorString(e));
        return AAFWI_ERR_CUDA;
    }
    return AAFWI_OK;
}

}  // extern "C"
