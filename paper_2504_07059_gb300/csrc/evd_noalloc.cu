// evd_noalloc.cu -- per-species mass of a population array without any
// allocation, for callers that cannot call cudaMalloc.
//
// It is a variant of the library's fixed-order mass reduction (block
// partials, then one block summing them in a fixed order).  The partials
// live in the file-scope device array below instead of memory obtained from
// cudaMalloc.  Host code must not pass the array's name to a kernel: on the
// host that name is only a stand-in, not a device address.  The device
// address is looked up with cudaGetSymbolAddress, with the device current,
// on the first call in each CUDA context of a device, and cached for that
// context: a context torn down and created again (cudaDeviceReset, a new
// primary context) loads the module afresh, so the address is looked up again.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "evd.h"
#include "evd_internal.h"

namespace {

constexpr int NA_BLOCK = 256;
constexpr int NA_MAX_BLOCKS = 1024;                 // grid-stride beyond this
constexpr int NA_MAX_SPECIES = 3;                  // the scratch holds partials for 3 species
constexpr int NA_MAX_DEVICES = 64;

std::mutex g_na_mutex;
// cached device address per device, valid for the context it was resolved in
double* g_na_scratch[NA_MAX_DEVICES] = {};
CUcontext g_na_ctx[NA_MAX_DEVICES] = {};

}  // namespace

// Partial sums, [block][species]: 1024 x 3 doubles = 24 KiB on every device
// that loads the library, held until the process exits.  Every call overwrites
// the slots it uses before reading them, so nothing needs clearing.
static __device__ __align__(256) double evd_noalloc_partials[NA_MAX_BLOCKS * NA_MAX_SPECIES];

__global__ void __launch_bounds__(NA_BLOCK)
evd_k_noalloc_mass_partial(const double* __restrict__ f, int ns, int q, long long nsites,
                           double* __restrict__ part)
{
    __shared__ double sm[NA_BLOCK / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long stride = (long long)gridDim.x * NA_BLOCK;
    for (int i = 0; i < ns; ++i) {
        double acc = 0.0;
        for (long long s = (long long)blockIdx.x * NA_BLOCK + threadIdx.x; s < nsites; s += stride)
            for (int a = 0; a < q; ++a) acc += f[((long long)i * q + a) * nsites + s];
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if (lane == 0) sm[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < NA_BLOCK / 32; ++w) t += sm[w];
            part[blockIdx.x * ns + i] = t;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
evd_k_noalloc_mass_finish(const double* __restrict__ part, int nblocks, int ns, double* __restrict__ out)
{
    __shared__ double sm[256];
    for (int i = 0; i < ns; ++i) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += 256) s += part[b * ns + i];
        sm[threadIdx.x] = s;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[i] = sm[0];
        __syncthreads();
    }
}

namespace {

// The driver's cuCtxGetCurrent, through the runtime's entry-point query (the
// library links the runtime only).
cudaError_t current_context(CUcontext* ctx)
{
    static PFN_cuCtxGetCurrent_v4000 get = nullptr;
    if (!get) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        get = (PFN_cuCtxGetCurrent_v4000)fn;
    }
    return get(ctx) == CUDA_SUCCESS ? cudaSuccess : cudaErrorContextIsDestroyed;
}

// Device address of the partials on the current device: resolved with that
// device current on the first call in its current context, cached for that
// context afterwards.
cudaError_t scratch_address(int dev, double** out)
{
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    CUcontext ctx = nullptr;
    cudaError_t e = current_context(&ctx);
    if (e != cudaSuccess) return e;
    if (!ctx || !g_na_scratch[dev] || g_na_ctx[dev] != ctx) {
        // the lookup also makes the runtime bind the device's primary
        // context where none is current yet; the context is read after it
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, evd_noalloc_partials);
        if (e != cudaSuccess) return e;
        e = current_context(&ctx);
        if (e != cudaSuccess) return e;
        g_na_scratch[dev] = (double*)p;
        g_na_ctx[dev] = ctx;
    }
    *out = g_na_scratch[dev];
    return cudaSuccess;
}

evd_status na_fail(evd_status s, const std::string& msg)
{
    evd::set_thread_error(msg);
    return s;
}

}  // namespace

extern "C" evd_status evd_population_mass_noalloc(const double* f_dev, int n_species, int q,
                                                  long long nsites, double* m_dev, void* cuda_stream)
{
    if (!f_dev || !m_dev) return na_fail(EVD_ERR_ARG, "f_dev and m_dev must not be NULL");
    if (n_species < 1 || n_species > NA_MAX_SPECIES)
        return na_fail(EVD_ERR_ARG, "n_species must be 1..3 (the scratch holds partials for 3 species)");
    if (q != 9 && q != 19) return na_fail(EVD_ERR_ARG, "q must be 9 (D2Q9) or 19 (D3Q19)");
    if (nsites < 1 || nsites > (1LL << 40)) return na_fail(EVD_ERR_ARG, "nsites must be 1 .. 2^40");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(EVD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    double* part = nullptr;
    e = scratch_address(dev, &part);
    if (e != cudaSuccess)
        return na_fail(EVD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    const long long want = (nsites + NA_BLOCK - 1) / NA_BLOCK;
    const int nblocks = (int)(want < NA_MAX_BLOCKS ? want : NA_MAX_BLOCKS);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    evd_k_noalloc_mass_partial<<<nblocks, NA_BLOCK, 0, st>>>(f_dev, n_species, q, nsites, part);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        evd_k_noalloc_mass_finish<<<1, 256, 0, st>>>(part, nblocks, n_species, m_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return na_fail(EVD_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return EVD_OK;
}
