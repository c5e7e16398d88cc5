// diag.cu -- diagnostics of the library, not steps of the method:
//   - measured FP64 and FP32 FMA throughput of the current GPU (the
//     denominators of the benchmark's roofline for the arithmetic-bound RHS
//     kernels);
//   - the kernels' FP64 arithmetic helpers (reciprocal, square root, tau^gamma,
//     e^(1/gamma)) and CUDA's own functions evaluated on caller arrays, so
//     that tests can bound their errors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/oct_hydro.h"
#include "oct_common.cuh"

oct_status octh_fail_text(oct_status st, const char *msg);  // oct_hydro.cu: sets oct_hydro_last_error

namespace {

// Written only when the chains reach a value they never reach (a fixed point
// near 1 is approached from below), so the compiler must keep every FMA.
__device__ double g_peak_sink;

// ILP independent FMA chains per thread, iters steps each: x <- x a + b.
template <class T, int ILP>
__global__ void __launch_bounds__(256) fma_chains(T a, T b, int iters)
{
    T x[ILP];
#pragma unroll
    for (int i = 0; i < ILP; i++)
        x[i] = (T)(threadIdx.x & 31) * (T)1e-3 + (T)i * (T)1e-2;
    for (int k = 0; k < iters; k++) {
#pragma unroll
        for (int i = 0; i < ILP; i++)
            x[i] = fma(x[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < ILP; i++)
        s += x[i];
    if (s == (T)-1)
        g_peak_sink = (double)s;
}

constexpr int ILP = 8;
constexpr int THREADS = 256;

// Flop rate (an FMA counts as two) of fma_chains<T> on a full grid (8 CTAs of
// 256 threads per SM), timed with CUDA events on stream s; iters grows until
// one launch takes at least target_ms.
template <class T>
cudaError_t measure(int n_sm, double target_ms, cudaStream_t s, double *flops)
{
    const int grid = n_sm * 8;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess)
        return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    const T a = (T)0.999, b = (T)1e-3;
    int iters = 1024;
    float ms = 0.f;
    for (int round = 0; round < 12; round++) {
        fma_chains<T, ILP><<<grid, THREADS, 0, s>>>(a, b, iters);  // warm-up of this size
        cudaEventRecord(e0, s);
        fma_chains<T, ILP><<<grid, THREADS, 0, s>>>(a, b, iters);
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess)
            break;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
            break;
        if (ms >= target_ms || iters >= (1 << 26))
            break;
        const double grow = ms > 0.f ? std::min(64.0, 1.2 * target_ms / ms) : 64.0;
        iters = (int)std::min<double>(1 << 26, std::ceil(iters * std::max(2.0, grow)));
    }
    if (e == cudaSuccess)
        e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess)
        *flops = 2.0 * ILP * (double)grid * THREADS * (double)iters / (ms * 1e-3);
    return e;
}

}  // namespace

extern "C" oct_status oct_hydro_pipe_peaks(double target_ms, double *fp64_tflops, double *fp32_tflops,
                                           void *cuda_stream)
{
    if (!fp64_tflops || !fp32_tflops)
        return octh_fail_text(OCT_E_ARG, "output pointers must not be NULL");
    if (!(target_ms > 0.0) || target_ms > 10000.0)
        return octh_fail_text(OCT_E_ARG, "target_ms must be in (0, 10000]");
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return octh_fail_text(OCT_E_CUDA, "no CUDA device");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double f64 = 0.0, f32 = 0.0;
    if (measure<double>(n_sm, target_ms, s, &f64) != cudaSuccess ||
        measure<float>(n_sm, target_ms, s, &f32) != cudaSuccess)
        return octh_fail_text(OCT_E_CUDA, "FMA throughput loop failed");
    *fp64_tflops = f64 / 1e12;
    *fp32_tflops = f32 / 1e12;
    return OCT_OK;
}

namespace {
// y[i] = fn(x[i]): 0 the kernels' reciprocal, 1 their square root, 2 their
// tau^gamma, 3 their e^(1/gamma); 16..19 the same with CUDA's own 1.0 / x,
// sqrt(x), pow(x, gamma) and pow(x, 1.0 / gamma).
__global__ void eval_math_kernel(int which, const double *x, double *y, long long n, double gamma)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        double r;
        switch (which) {
        case 0: r = octh::rcp_nr(v); break;
        case 1: r = octh::sqrt_nr(v); break;
        case 2: r = octh::eint_of_tau(v, gamma); break;
        case 3: r = octh::tau_of_eint(v, gamma); break;
        case 16: r = 1.0 / v; break;
        case 17: r = sqrt(v); break;
        case 18: r = pow(v, gamma); break;
        default: r = pow(v, 1.0 / gamma); break;
        }
        y[i] = r;
    }
}
}  // namespace

extern "C" oct_status oct_hydro_eval_math(int which, const double *x, double *y, int64_t n, double gamma,
                                          void *cuda_stream)
{
    if (!((which >= 0 && which <= 3) || (which >= 16 && which <= 19)))
        return octh_fail_text(OCT_E_ARG, "which must be 0..3 or 16..19");
    if (!x || !y || n < 0)
        return octh_fail_text(OCT_E_ARG, "x and y must not be NULL and n must be >= 0");
    if (n == 0)
        return OCT_OK;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    eval_math_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)cuda_stream>>>(which, x, y, n, gamma);
    if (cudaGetLastError() != cudaSuccess)
        return octh_fail_text(OCT_E_CUDA, "eval_math launch failed");
    return OCT_OK;
}
