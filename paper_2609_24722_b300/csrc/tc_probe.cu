// tc_probe.cu -- pipe-throughput probes for the roofline of the pair kernels.
//
// The pair kernels are bound by instruction pipes, not by memory: the mixed
// form by the float32 FMA pipe and the MUFU (special function) unit, the
// float64 form by the float64 pipe.  These probes run long chains of
// independent FFMA, DFMA and MUFU.RSQ instructions on every SM and report the
// achieved operation rates, which the benchmark uses as peaks.
#include "tc_internal.h"

namespace tc {
namespace {

constexpr int kChains = 8;

__global__ void k_probe_ffma(float b, float c, int iters, float* sink)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-3f + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 1234.5f) *sink = s;
}

__global__ void k_probe_dfma(double b, double c, int iters, double* sink)
{
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-3 + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 1234.5) *sink = s;
}

__global__ void k_probe_mufu(int iters, float* sink)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-3f + k + 1.0f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            float y;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[k]));
            a[k] = y;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 1234.5f) *sink = s;
}

// The far-tile pair mix of the mixed pass with no memory traffic: per step and
// chain, two packed differences, r^2 as a packed mul + fma, two MUFU.RSQ, r^-3
// as two packed muls and two packed gradient fmas (2 pairs).  The sources
// move by a packed add per step shared by all chains.
__global__ void k_probe_pairmix(int iters, float* sink)
{
    constexpr int K = 4;
    float2 x[K], y[K], gx[K], gy[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        x[k] = make_float2(0.1f * k + threadIdx.x * 1e-4f, 0.2f + 0.1f * k);
        y[k] = make_float2(0.3f - 0.05f * k, 0.15f * k + 0.01f);
        gx[k] = gy[k] = make_float2(0.f, 0.f);
    }
    float2 qx = make_float2(-0.7f, -0.69f), qy = make_float2(0.4f, 0.41f);
    const float2 dq = make_float2(1e-7f, -1e-7f);
    for (int it = 0; it < iters; ++it) {
        qx = __fadd2_rn(qx, dq);
        qy = __fadd2_rn(qy, dq);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float2 dx = __fadd2_rn(x[k], qx);
            const float2 dy = __fadd2_rn(y[k], qy);
            const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
            float a, b;
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(a) : "f"(r2.x));
            asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(b) : "f"(r2.y));
            const float2 inv = make_float2(a, b);
            const float2 inv3 = __fmul2_rn(__fmul2_rn(inv, inv), inv);
            gx[k] = __ffma2_rn(dx, inv3, gx[k]);
            gy[k] = __ffma2_rn(dy, inv3, gy[k]);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) s += gx[k].x + gx[k].y + gy[k].x + gy[k].y;
    if (s == 1234.5f) *sink = s;
}

template <class F> double time_ms(F launch, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int reps)
{
    launch();  // warm-up
    double best = 1e30;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    return best;
}

}  // namespace
}  // namespace tc

extern "C" tc_status tc_probe_pipes(double* rates, tc_stream stream)
{
    if (!rates) return TC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int sms = tc::sm_count();
    const int threads = 256, blocks = sms * 8;
    const double nthr = (double)threads * blocks;
    float* sink = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return TC_ERR_NO_MEMORY;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int it32 = 8192, it64 = 256, itmu = 2048;
    double ms_f = tc::time_ms([&] { tc::k_probe_ffma<<<blocks, threads, 0, s>>>(1.0000001f, 1e-7f, it32, sink); }, s, e0, e1, 5);
    double ms_d = tc::time_ms([&] { tc::k_probe_dfma<<<blocks, threads, 0, s>>>(1.0000000001, 1e-9, it64, (double*)sink); }, s, e0, e1, 5);
    double ms_m = tc::time_ms([&] { tc::k_probe_mufu<<<blocks, threads, 0, s>>>(itmu, sink); }, s, e0, e1, 5);
    const int itpm = 1024;
    double ms_p = tc::time_ms([&] { tc::k_probe_pairmix<<<blocks, threads, 0, s>>>(itpm, sink); }, s, e0, e1, 5);
    cudaError_t e = cudaGetLastError();
    rates[0] = nthr * it32 * tc::kChains / (ms_f * 1e-3);  // FFMA lane operations / s
    rates[1] = nthr * it64 * tc::kChains / (ms_d * 1e-3);  // DFMA operations / s
    rates[2] = nthr * itmu * tc::kChains / (ms_m * 1e-3);  // MUFU.RSQ operations / s
    rates[3] = nthr * itpm * 4 * 2 / (ms_p * 1e-3);        // far-tile pair mix: ordered pairs / s
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return e == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}
