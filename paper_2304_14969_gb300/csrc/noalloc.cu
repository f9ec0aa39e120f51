// Inner product <a|b> that allocates nothing.
//
// qsim_inner_product keeps its partial sums in per-state scratch that the
// library allocates with cudaMalloc. Some callers cannot let the library
// allocate: a host program that has handed all device memory to another
// framework's allocator, or a loop with a latency budget that must not
// stall in the driver's allocator, still needs <a|b> of two kets it already
// owns. This variant keeps its scratch in one file-scope __device__ array
// of fixed size instead, so a call performs no cudaMalloc, cudaFree or
// allocating library routine; the caller passes the two kets and a host
// buffer for the result.
//
// The array holds kNaRows partial rows of two doubles plus the two FP64
// results (16.4 KB on every GPU that loads the library, held until exit).
// Every call writes each partial row that it later reads, so nothing has to
// be cleared between calls. All calls share the array: two calls whose
// kernels overlap on the GPU (different streams, or host threads without
// ordering) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "qsim_internal.h"

namespace qs {

static const int kNaRows = 1024;        // partial rows = CTAs of the sum kernel
static const int kNaThreads = 256;
static const int kNaMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[2 * kNaRows + 2];

template <typename R> struct NaV;
template <> struct NaV<float> { using T = float2; };
template <> struct NaV<double> { using T = double2; };

// One row per CTA: the CTA's FP64 sum of conj(a_i) b_i (runs of 8 terms
// summed in the ket's precision first).
template <typename R>
__global__ void __launch_bounds__(kNaThreads) k_na_inner(const typename NaV<R>::T *__restrict__ a,
                                                         const typename NaV<R>::T *__restrict__ b, uint64_t N,
                                                         double *__restrict__ rows)
{
    double re = 0, im = 0;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x * 8;
    for (uint64_t base = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8; base < N; base += stride) {
        R sr = 0, si = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            if (base + j < N) {
                auto x = a[base + j];
                auto y = b[base + j];
                sr = fma(x.x, y.x, fma(x.y, y.y, sr));
                si = fma(x.x, y.y, fma(-x.y, y.x, si));
            }
        }
        re += (double)sr;
        im += (double)si;
    }
    __shared__ double sh[2][kNaThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = re;
        sh[1][threadIdx.x >> 5] = im;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0;
        for (int w = 0; w < kNaThreads / 32; w++) s += sh[threadIdx.x][w];
        rows[2 * blockIdx.x + threadIdx.x] = s;
    }
}

__global__ void k_na_final(const double *__restrict__ rows, int nrows, double *__restrict__ out)
{
    if (threadIdx.x < 2) {
        double s = 0;
        for (int r = 0; r < nrows; r++) s += rows[2 * r + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Device address of the scratch array, looked up once per device with that
// device current (the host-side name of a __device__ variable is only a
// stand-in, not an address a kernel can use).
static double *scratch_for_current_device(qsim_status *st)
{
    static std::mutex mu;
    static double *ptr[kNaMaxDevices] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *st = cuda_fail(e, "cudaGetDevice");
        return nullptr;
    }
    if (dev < 0 || dev >= kNaMaxDevices) {
        *st = fail(QSIM_E_UNSUPPORTED, "device %d beyond the %d devices this entry point supports", dev,
                   kNaMaxDevices);
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            *st = cuda_fail(e, "cudaGetSymbolAddress (inner-product scratch)");
            return nullptr;
        }
        ptr[dev] = (double *)p;
    }
    *st = QSIM_OK;
    return ptr[dev];
}

}  // namespace qs

using namespace qs;

extern "C" qsim_status qsim_inner_product_noalloc(const void *a_dev, const void *b_dev, int n, qsim_dtype dt,
                                                  void *stream, double out[2])
{
    clear_error();
    if (!a_dev || !b_dev || !out) return fail(QSIM_E_INVAL, "a_dev, b_dev and out must not be NULL");
    if (dt != QSIM_C64 && dt != QSIM_C128) return fail(QSIM_E_INVAL, "unknown dtype %d", (int)dt);
    if (n < 1 || n > 36)
        return fail(QSIM_E_INVAL, "n=%d outside [1, 36]: the fixed scratch serves kets of at most 2^36 amplitudes",
                    n);
    qsim_status st = QSIM_OK;
    double *scr = scratch_for_current_device(&st);
    if (!scr) return st;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t N = 1ull << n;
    uint64_t items = (N + 7) / 8;
    int rows = (int)std::max<uint64_t>(1, std::min<uint64_t>((items + kNaThreads - 1) / kNaThreads, kNaRows));
    if (dt == QSIM_C64)
        k_na_inner<float><<<rows, kNaThreads, 0, s>>>((const float2 *)a_dev, (const float2 *)b_dev, N, scr);
    else
        k_na_inner<double><<<rows, kNaThreads, 0, s>>>((const double2 *)a_dev, (const double2 *)b_dev, N, scr);
    QS_CUDA(cudaGetLastError());
    k_na_final<<<1, 32, 0, s>>>(scr, rows, scr + 2 * kNaRows);
    QS_CUDA(cudaGetLastError());
    QS_CUDA(cudaMemcpyAsync(out, scr + 2 * kNaRows, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    QS_CUDA(cudaStreamSynchronize(s));
    return QSIM_OK;
}
