// xrd_unit_rates: issue rates of the arithmetic units that bound the
// structure-factor kernel (MUFU sin, cos and ex2, FP32 FMA) and of FP64 FMA
// (which the enumeration and output kernels keep off their hot loops), on the
// handle's device. One CTA of 1024 threads runs on one SM; every thread keeps
// eight independent chains of one operation in flight, and the SM's clock64
// counter times the loop, so the result is in lane operations per SM per
// clock, independent of the clock frequency. The structure-factor roofline of
// a batch follows from these rates and the batch's operation counts.
#include "xrd_launch.h"

namespace xrd {

constexpr int kRateThreads = 1024;
constexpr int kRateChains = 8;

template <int OP>
__global__ void __launch_bounds__(kRateThreads) k_unit_rate(int iters, float seed, float* __restrict__ sink,
                                                           long long* __restrict__ cycles)
{
    float x[kRateChains];
#pragma unroll
    for (int i = 0; i < kRateChains; i++) x[i] = seed + 1e-3f * (float)i + 1e-7f * (float)threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < kRateChains; i++) {
            if (OP == 0) x[i] = __sinf(x[i]);
            else if (OP == 1) x[i] = __cosf(x[i]);
            else if (OP == 2) x[i] = ex2_approx(-x[i]);
            else x[i] = fmaf(x[i], 0.999f, 1e-3f);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) *cycles = t1 - t0;
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < kRateChains; i++) acc += x[i];
    if (acc == 12345.f) sink[threadIdx.x] = acc;  // keeps the chains live; never true for these inputs
}

// The same loop with FP64 FMA chains.
__global__ void __launch_bounds__(kRateThreads) k_unit_rate_f64(int iters, double seed, double* __restrict__ sink,
                                                               long long* __restrict__ cycles)
{
    double x[kRateChains];
#pragma unroll
    for (int i = 0; i < kRateChains; i++) x[i] = seed + 1e-3 * (double)i + 1e-7 * (double)threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < kRateChains; i++) x[i] = fma(x[i], 0.999, 1e-3);
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) *cycles = t1 - t0;
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < kRateChains; i++) acc += x[i];
    if (acc == 12345.0) sink[threadIdx.x] = acc;
}

}  // namespace xrd

extern "C" int xrd_unit_rates(xrd_handle* h, double* rates)
{
    if (!h || !rates) return XRD_EINVAL;
    const int dev = xrd::handle_device(h);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return XRD_ECUDA;
    cudaStream_t st = nullptr;
    long long* d_cyc = nullptr;
    double* d_sink = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&d_cyc, 5 * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&d_sink, xrd::kRateThreads * sizeof(double));
    constexpr int kIters = 2048;
    if (e == cudaSuccess) {
        // a warm-up pass of each, then the timed pass
        for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
            float* fs = (float*)d_sink;
            xrd::k_unit_rate<0><<<1, xrd::kRateThreads, 0, st>>>(kIters, 0.5f, fs, d_cyc + 0);
            xrd::k_unit_rate<1><<<1, xrd::kRateThreads, 0, st>>>(kIters, 0.5f, fs, d_cyc + 1);
            xrd::k_unit_rate<2><<<1, xrd::kRateThreads, 0, st>>>(kIters, 0.5f, fs, d_cyc + 2);
            xrd::k_unit_rate<3><<<1, xrd::kRateThreads, 0, st>>>(kIters, 0.5f, fs, d_cyc + 3);
            xrd::k_unit_rate_f64<<<1, xrd::kRateThreads, 0, st>>>(kIters / 8, 0.5, d_sink, d_cyc + 4);
            e = cudaStreamSynchronize(st);
        }
    }
    long long cyc[5] = {0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(cyc, d_cyc, sizeof(cyc), cudaMemcpyDeviceToHost);
    if (d_cyc) cudaFree(d_cyc);
    if (d_sink) cudaFree(d_sink);
    if (st) cudaStreamDestroy(st);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess) return xrd::set_error(h, XRD_ECUDA, "xrd_unit_rates: CUDA call failed");
    const double ops = (double)xrd::kRateThreads * xrd::kRateChains * kIters;
    for (int i = 0; i < 5; i++) rates[i] = cyc[i] > 0 ? (i == 4 ? ops / 8 : ops) / (double)cyc[i] : 0.0;
    return XRD_OK;
}
