// bn_peak.cu -- measured CUDA-core FMA rates of the device (FP32 scalar, FP32 paired, FP64).
//
// The operator kernels are bound by the FP32 FMA pipe (mixed precision) or the FP64 FMA pipe
// (FP64 mode), so their roofline denominator is the rate at which this device retires
// independent FMA chains.  Each thread runs kChains independent chains of `iters` dependent
// multiply-adds; enough warps per SM hide the FMA latency, and the result is written out so that
// nothing is eliminated.  Timed with CUDA events around one launch after an untimed one.
#include <cstdint>
#include <string>

#include "bn_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_chain_f32(int iters, float a, float b, float* out) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// fma.rn.f32x2: one instruction, two FP32 multiply-adds
__global__ void __launch_bounds__(kThreads) k_chain_f32x2(int iters, float a, float b, float* out) {
    uint64_t x[kChains];
    const uint64_t av = bn::pack2(a, a), bv = bn::pack2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = bn::pack2((float)(threadIdx.x + c), (float)(threadIdx.x - c));
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = bn::fma2(x[c], av, bv);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float lo, hi;
        bn::split2(x[c], lo, hi);
        s += lo + hi;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_chain_f64(int iters, double a, double b, float* out) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

}  // namespace

extern "C" bn_status bn_measure_fma_peak(int kind, void* cuda_stream, double* out, size_t count) {
    if (!out || count < 3 || kind < 0 || kind > 2) {
        bn::set_last_error("bn_measure_fma_peak: kind in 0..2, out non-null, count >= 3");
        return BN_ERR_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        bn::set_last_error("bn_measure_fma_peak: no CUDA device");
        return BN_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // FP32 chains: 4 CTAs of 256 threads per SM; FP64 (1/64 of the FP32 rate): fewer iterations
    const int grid = 4 * sms;
    const int iters = kind == 2 ? 2048 : 65536;
    float* buf = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaMalloc(&buf, sizeof(float) * grid * kThreads);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        if (rep > 0) cudaEventRecord(t0, st);
        if (kind == 0) k_chain_f32<<<grid, kThreads, 0, st>>>(iters, 0.999999f, 1e-7f, buf);
        else if (kind == 1) k_chain_f32x2<<<grid, kThreads, 0, st>>>(iters, 0.999999f, 1e-7f, buf);
        else k_chain_f64<<<grid, kThreads, 0, st>>>(iters, 0.9999999999, 1e-12, buf);
        if (rep > 0) cudaEventRecord(t1, st);
        e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess && rep > 0) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, t0, t1);
            if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) {
        cudaGetLastError();
        bn::set_last_error(std::string("bn_measure_fma_peak: ") + cudaGetErrorString(e));
        return BN_ERR_CUDA;
    }
    const double flops = 2.0 * (kind == 1 ? 2.0 : 1.0) * kChains * (double)iters * grid * kThreads;
    out[0] = flops / (best * 1e-3) * 1e-12;
    out[1] = best;
    out[2] = flops;
    return BN_OK;
}
