// Triple-product sums without any device allocation.
//
// fbs_triple_sums_noalloc computes num[t] = sum_p f_a[p] f_b[p] f_c[p] for
// caller-supplied device fields and triplets.  It is the reduction the
// FP32 contraction performs (per-block FP64 partial sums, then a reduction
// in a fixed order), but its per-block partials live in the file-scope
// device array below instead of plan-owned memory, so the call allocates
// nothing.  It serves callers whose device memory is owned by someone else
// (a framework allocator that must account for every byte, or a process that
// reserves all device memory up front and forbids further cudaMalloc).
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "fbs_internal.h"

namespace fbs {

// Scratch: one FP64 partial per (block, triplet).  Every GPU that loads the
// library holds these 152 x 4096 x 8 B = 4.75 MiB until the process exits.
static constexpr int kNaBlocks = 152;
static constexpr int kNaMaxTrip = 4096;
static __device__ __align__(256) double g_noalloc_partials[kNaBlocks * kNaMaxTrip];

// Block j sums points [p0_j, p1_j) of every triplet and writes (not adds) its
// partial, so no entry needs clearing between calls.
__global__ void __launch_bounds__(256) noalloc_triple_kernel(const float *__restrict__ f,
                                                             long long bin_stride, long long npts,
                                                             int nfields,
                                                             const int32_t *__restrict__ abc, int ntrip,
                                                             double *__restrict__ part) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const long long p0 = npts * blockIdx.x / gridDim.x;
    const long long p1 = npts * (blockIdx.x + 1) / gridDim.x;
    for (int t = warp; t < ntrip; t += nw) {
        const int a = abc[3 * t], b = abc[3 * t + 1], c = abc[3 * t + 2];
        if (a < 0 || b < 0 || c < 0 || a >= nfields || b >= nfields || c >= nfields) {
            if (lane == 0) part[(long long)blockIdx.x * kNaMaxTrip + t] = __longlong_as_double(0x7ff8000000000000LL);
            continue;  // a field index outside the caller's array: NaN, no access
        }
        const float *fa = f + (long long)abc[3 * t] * bin_stride;
        const float *fb = f + (long long)abc[3 * t + 1] * bin_stride;
        const float *fc = f + (long long)abc[3 * t + 2] * bin_stride;
        double acc = 0.0;
        float s = 0.f;
        int n = 0;
        for (long long p = p0 + lane; p < p1; p += 32) {
            s = fmaf(fa[p] * fb[p], fc[p], s);
            if (++n == 64) {  // FP32 runs of 64 terms, FP64 across runs
                acc += (double)s;
                s = 0.f;
                n = 0;
            }
        }
        acc += (double)s;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) part[(long long)blockIdx.x * kNaMaxTrip + t] = acc;
    }
}

__global__ void noalloc_reduce_kernel(const double *__restrict__ part, int rows, int ntrip,
                                      double *__restrict__ num) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntrip) return;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s += part[(long long)r * kNaMaxTrip + t];
    num[t] = s;
}

// Device address of the scratch array, looked up once per device with that
// device current (a host-side symbol name is not a device address).
static std::mutex g_na_mu;
static double *g_na_ptr[64];

static cudaError_t noalloc_scratch(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

}  // namespace fbs

extern "C" fbs_status fbs_triple_sums_noalloc(const float *fields, int nfields, long long bin_stride,
                                              long long npts, const int32_t *abc, int ntrip, double *num,
                                              void *cuda_stream) {
    using namespace fbs;
    if (!fields || !abc || !num || nfields < 1 || npts < 0 || bin_stride < npts || ntrip < 0) {
        set_error("fbs_triple_sums_noalloc: bad argument");
        return FBS_ERR_ARG;
    }
    if (ntrip > kNaMaxTrip) {
        set_error("fbs_triple_sums_noalloc: ntrip " + std::to_string(ntrip) + " exceeds the maximum " +
                  std::to_string(kNaMaxTrip));
        return FBS_ERR_ARG;
    }
    if (ntrip == 0) return FBS_OK;
    double *part = nullptr;
    cudaError_t e = noalloc_scratch(&part);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("fbs_triple_sums_noalloc: scratch lookup failed: ") + cudaGetErrorString(e));
        return FBS_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    noalloc_triple_kernel<<<kNaBlocks, 256, 0, s>>>(fields, bin_stride, npts, nfields, abc, ntrip, part);
    noalloc_reduce_kernel<<<(ntrip + 255) / 256, 256, 0, s>>>(part, kNaBlocks, ntrip, num);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("fbs_triple_sums_noalloc: launch failed: ") + cudaGetErrorString(e));
        return FBS_ERR_CUDA;
    }
    return FBS_OK;
}
