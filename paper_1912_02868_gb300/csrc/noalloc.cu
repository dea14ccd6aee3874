// True-residual norms of the Wilson-Dirac system with no device allocation.
//
// The solver's stopping test (Section 2: outer FGMRES stops when
// ||b - D x|| <= tol ||b||) is computed inside the library from workspaces the
// handle allocated at set-up.  Some callers hold no handle and may not allocate
// device memory at all: an HMC or measurement driver that owns every byte of
// HBM through its own pool and checks a solution between trajectories, or a
// monitoring thread that must not call cudaMalloc/cudaFree while other streams
// run (both can synchronise the whole device, and a cudaMalloc can fail under a
// full pool).  This entry point serves them: the residual goes to a buffer the
// caller owns, and the two reductions use a fixed scratch array that lives in
// the module image (a file-scope __device__ array), sized for lattices of up to
// 1024 x 1024 sites.
//
// Set-up: the first call on each device (with that device current) looks up
// the array's address with cudaGetSymbolAddress and caches it.  That first call
// should come before any stream capture on the device begins.
//
// The scratch is one per device: calls whose kernels can overlap on the GPU
// (other streams, other host threads) race on it and must be serialised.
#include <cmath>
#include <initializer_list>
#include <mutex>

#include "ops.cuh"

namespace mg {

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 4;                                // elements per thread (one block: 1024)
constexpr int NA_MAX_BLOCKS = 2048;                             // partial sums held by the scratch
constexpr long NA_MAX_N = (long)NA_MAX_BLOCKS * NA_THREADS * NA_PER_THREAD;  // 2^21 complex entries
constexpr long NA_MAX_SITES = NA_MAX_N / 2;                     // 2 spin components per site
constexpr int NA_MAX_DEVICES = 64;

// [0, NA_MAX_BLOCKS): per-block (||r||^2, ||b||^2) partials, each written by
// its block before it is read; [NA_MAX_BLOCKS]: the totals; the first word of
// [NA_MAX_BLOCKS + 1]: the arrival counter of the blocks, which must be zero
// when a launch starts (cleared by every call).  (2048 + 2) x 16 bytes =
// 32 800 bytes in all.
static __device__ __align__(256) double2 na_scratch[NA_MAX_BLOCKS + 2];

std::mutex na_mutex;
double2* na_ptr[NA_MAX_DEVICES] = {};

mg_status scratch_of_current_device(double2** out) {
    int dev = 0;
    MG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        set_error("device ordinal %d is beyond the %d devices the residual scratch tracks", dev, NA_MAX_DEVICES);
        return MG_EINVAL;
    }
    std::lock_guard<std::mutex> lock(na_mutex);
    if (!na_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the residual scratch failed on device %d: %s", dev,
                      cudaGetErrorString(e));
            return MG_ECUDA;
        }
        na_ptr[dev] = static_cast<double2*>(p);
    }
    *out = na_ptr[dev];
    return MG_OK;
}

// ||r||^2 and ||b||^2 in FP64: block i sums elements [1024 i, 1024 (i + 1)) in a
// fixed order, the last block to arrive adds the block partials in block order.
__global__ void __launch_bounds__(NA_THREADS) k_residual_norms(const double2* __restrict__ r,
                                                               const double2* __restrict__ b, long n,
                                                               double2* scratch) {
    __shared__ double2 sm[NA_THREADS / 32];
    __shared__ bool am_last;
    double2* part = scratch;
    double2* total = scratch + NA_MAX_BLOCKS;
    unsigned* arrivals = reinterpret_cast<unsigned*>(scratch + NA_MAX_BLOCKS + 1);
    const long base = (long)blockIdx.x * NA_THREADS * NA_PER_THREAD + threadIdx.x;
    double rr = 0.0, bb = 0.0;
#pragma unroll
    for (int u = 0; u < NA_PER_THREAD; ++u) {
        const long e = base + (long)u * NA_THREADS;
        if (e < n) {
            const double2 re = r[e], be = b[e];
            rr += re.x * re.x + re.y * re.y;
            bb += be.x * be.x + be.y * be.y;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
        bb += __shfl_xor_sync(0xffffffffu, bb, o);
    }
    if (lane == 0) sm[warp] = make_double2(rr, bb);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 s = make_double2(0.0, 0.0);
        for (int w = 0; w < NA_THREADS / 32; ++w) {
            s.x += sm[w].x;
            s.y += sm[w].y;
        }
        part[blockIdx.x] = s;
        __threadfence();
        am_last = atomicAdd(arrivals, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!am_last || warp != 0) return;
    __threadfence();
    double2 s = make_double2(0.0, 0.0);
    for (unsigned i = lane; i < gridDim.x; i += 32) {
        const double2 p = __ldcg(part + i);
        s.x += p.x;
        s.y += p.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    }
    if (lane == 0) {
        *total = s;
        *arrivals = 0u;
    }
}

}  // namespace

}  // namespace mg

using namespace mg;

extern "C" {

mg_status mg_wilson_residual_noalloc(const void* gauge, int L_x, int L_t, double m0, const void* b, const void* x,
                                     void* r, double* norms, void* stream) {
    if (!gauge || !b || !x || !r || !norms)
        return set_error("gauge, b, x, r and norms must be non-NULL"), MG_EINVAL;
    if (r == x || r == b) return set_error("r must not alias x or b"), MG_EINVAL;
    if (L_x < 2 || L_t < 2) return set_error("lattice extents must be >= 2"), MG_EINVAL;
    const long sites = (long)L_x * L_t;
    if (sites > NA_MAX_SITES) {
        set_error("lattice of %d x %d sites exceeds the fixed residual scratch (at most %ld sites)", L_x, L_t,
                  NA_MAX_SITES);
        return MG_EINVAL;
    }
    int cur = 0;
    MG_CUDA_TRY(cudaGetDevice(&cur));
    for (const void* p : {gauge, b, x, static_cast<const void*>(r)}) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            (void)cudaGetLastError();
            return set_error("gauge, b, x and r must be device pointers"), MG_EINVAL;
        }
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
            return set_error("gauge, b, x and r must be device pointers"), MG_EINVAL;
        // the scratch address and the kernels belong to the current device
        if (a.type == cudaMemoryTypeDevice && a.device != cur)
            return set_error("gauge, b, x and r must be memory of the current device (%d)", cur), MG_EINVAL;
    }
    double2* scratch = nullptr;
    MG_TRY(scratch_of_current_device(&scratch));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long n = 2 * sites;
    // r = b - D x (the solver's own FP64 residual kernel)
    launch_wilson<double>(static_cast<double2*>(r), static_cast<const double2*>(x), static_cast<const double2*>(gauge),
                          static_cast<const double2*>(b), m0, L_x, L_t, false, Gate{}, s);
    MG_LAUNCH_CHECK();
    MG_CUDA_TRY(cudaMemsetAsync(scratch + NA_MAX_BLOCKS + 1, 0, sizeof(double2), s));
    const unsigned blocks = (unsigned)((n + NA_THREADS * NA_PER_THREAD - 1) / (NA_THREADS * NA_PER_THREAD));
    k_residual_norms<<<blocks, NA_THREADS, 0, s>>>(static_cast<const double2*>(r), static_cast<const double2*>(b), n,
                                                   scratch);
    count_launch();
    MG_LAUNCH_CHECK();
    double2 tot;
    MG_CUDA_TRY(cudaMemcpyAsync(&tot, scratch + NA_MAX_BLOCKS, sizeof(double2), cudaMemcpyDeviceToHost, s));
    MG_CUDA_TRY(cudaStreamSynchronize(s));
    norms[0] = std::sqrt(tot.x);
    norms[1] = std::sqrt(tot.y);
    return MG_OK;
}

}  // extern "C"
