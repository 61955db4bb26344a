// Pair-distance histogram that allocates nothing (espp_rdf_counts_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs inside a framework
// which reserved the device memory up front and hands out only its own pool,
// and latency-critical loops that cannot take the implicit device
// synchronisation of cudaMalloc/cudaFree.  For them this file keeps the
// histogram's working buffer in a fixed file-scope device array instead of
// memory allocated per handle.  The array (ESPP_NOALLOC_MAX_BINS counters,
// 32 KiB) is part of the module image: every GPU that loads the library holds
// it until the process exits.
#include <mutex>

#include "common.cuh"

namespace espp {

static __device__ __align__(256) unsigned long long g_rdf_scratch[ESPP_NOALLOC_MAX_BINS];

// The same histogram as the handle-based path (unique pairs i < j, minimum
// image, integer counts), reading caller-owned double positions in id order.
__global__ void __launch_bounds__(256) k_rdf_noalloc(const double* __restrict__ x, int n, double L0,
                                                     double L1, double L2, double rmax2,
                                                     double inv_dr, int nbins,
                                                     unsigned long long* __restrict__ scratch) {
    extern __shared__ unsigned int hist[];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const double H0 = 0.5 * L0, H1 = 0.5 * L1, H2 = 0.5 * L2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double ax = x[3 * (size_t)i], ay = x[3 * (size_t)i + 1], az = x[3 * (size_t)i + 2];
        for (int j = i + 1; j < n; ++j) {
            const double dx = min_image(ax, x[3 * (size_t)j], L0, H0);
            const double dy = min_image(ay, x[3 * (size_t)j + 1], L1, H1);
            const double dz = min_image(az, x[3 * (size_t)j + 2], L2, H2);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < rmax2) {
                int b = (int)(sqrt(r2) * inv_dr);
                if (b >= nbins) b = nbins - 1;
                atomicAdd(&hist[b], 1u);
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (hist[b]) atomicAdd(&scratch[b], (unsigned long long)hist[b]);
}

__global__ void k_rdf_noalloc_finish(const unsigned long long* __restrict__ scratch, int nbins,
                                     int64_t* __restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbins) out[b] = (int64_t)scratch[b];
}

// Device address of the scratch array, looked up once per device with that
// device current.
static std::mutex g_scratch_mu;
static unsigned long long* g_scratch_ptr[64] = {nullptr};

static cudaError_t scratch_for_current_device(unsigned long long** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_rdf_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = reinterpret_cast<unsigned long long*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace espp

extern "C" int espp_rdf_counts_noalloc(const double* x_device, int64_t n, const double box[3],
                                       double rmax, int32_t nbins, int64_t* counts_device,
                                       void* cuda_stream) {
    // n is bounded like the handle path's all-pairs histogram: the O(n^2)
    // kernel would otherwise hold the GPU for minutes on a large system
    if (!x_device || !counts_device || !box || n < 0 || n > ESPP_NOALLOC_MAX_N) return ESPP_ERR_ARG;
    if (nbins < 1 || nbins > ESPP_NOALLOC_MAX_BINS) return ESPP_ERR_ARG;
    for (int c = 0; c < 3; ++c)
        if (!(box[c] > 0) || !(rmax > 0) || !(rmax < 0.5 * box[c])) return ESPP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned long long* scratch = nullptr;
    if (espp::scratch_for_current_device(&scratch) != cudaSuccess) return ESPP_ERR_CUDA;
    // the array keeps the previous call's counts: clear the part this call uses
    if (cudaMemsetAsync(scratch, 0, (size_t)nbins * sizeof(unsigned long long), st) != cudaSuccess)
        return ESPP_ERR_CUDA;
    if (n > 1) {
        espp::k_rdf_noalloc<<<4 * espp::sm_count(), 256, sizeof(unsigned int) * nbins, st>>>(
            x_device, (int)n, box[0], box[1], box[2], rmax * rmax, nbins / rmax, nbins, scratch);
    }
    espp::k_rdf_noalloc_finish<<<(nbins + 255) / 256, 256, 0, st>>>(scratch, nbins, counts_device);
    return cudaGetLastError() == cudaSuccess ? ESPP_OK : ESPP_ERR_CUDA;
}
