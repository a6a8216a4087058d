// Measurement helpers of the benchmark (include/mp_probe.h): the rate of
// random 32-byte sector reads and the FMA throughput of this GPU, the ceilings
// the likelihood kernel's rooflines are read against.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../../include/megaparticles.h"
#include "../../../include/mp_probe.h"

namespace {

constexpr int PR_THREADS = 256;
constexpr int PR_LANES = 16;   // independent reads in flight per thread

__global__ void __launch_bounds__(PR_THREADS) k_probe_reads(const uint32_t* __restrict__ words, uint64_t n_words,
                                                            int rounds, uint32_t seed, uint32_t* __restrict__ sink) {
    const uint32_t tid = blockIdx.x * PR_THREADS + threadIdx.x;
    uint32_t x[PR_LANES];
#pragma unroll
    for (int u = 0; u < PR_LANES; ++u) x[u] = (tid * PR_LANES + u) * 2654435761u ^ seed;
    uint32_t acc = 0;
    for (int r = 0; r < rounds; ++r) {
        uint32_t v[PR_LANES];
        // all 16 addresses first (LCG, Numerical Recipes constants), then the
        // 16 loads, then their use: 16 reads per thread in flight
#pragma unroll
        for (int u = 0; u < PR_LANES; ++u) {
            x[u] = x[u] * 1664525u + 1013904223u;
            v[u] = __ldg(words + (((uint64_t)x[u] * n_words) >> 32));   // uniform in [0, n_words)
        }
#pragma unroll
        for (int u = 0; u < PR_LANES; ++u) acc += v[u];
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;   // keeps the reads live; practically never taken
}

// 16 independent chains a = a * m + c per thread (|m| < 1 keeps them bounded)
template <typename T>
__global__ void __launch_bounds__(PR_THREADS) k_probe_fma(int iters, T m, T c, T* __restrict__ sink) {
    T a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = (T)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; ++k) a[k] = fma(a[k], m, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += a[k];
    if (s == (T)-1.2345) sink[0] = s;
}

__global__ void __launch_bounds__(PR_THREADS) k_probe_fma2(int iters, float m, float c, float* __restrict__ sink) {
    float2 a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x - k));
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], m2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k].x + a[k].y;
    if (s == -1.2345f) sink[0] = s;
}

bool device_ptr(const void* p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

// Runs launch() once untimed and `repeats` times between two events.
template <typename F>
int timed(F launch, int repeats, cudaStream_t s, float* ms_out) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MP_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = MP_ECUDA;
    if (rc == MP_OK) {
        launch(0);
        cudaEventRecord(e0, s);
        for (int r = 0; r < repeats; ++r) launch(r + 1);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            rc = MP_ECUDA;
        *ms_out = ms / repeats;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" int mp_probe_random_reads(const uint32_t* words, int64_t n_words, int blocks, int reads_per_thread,
                                     int repeats, void* cuda_stream, float* ms_out, int64_t* reads_out) {
    if (!words || !ms_out || n_words < 1 || n_words > ((int64_t)1 << 32) || blocks < 1 || reads_per_thread < 1 ||
        repeats < 1 || !device_ptr(words))
        return MP_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int rounds = (reads_per_thread + PR_LANES - 1) / PR_LANES;
    uint32_t* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(uint32_t)) != cudaSuccess) return MP_ECUDA;
    const int rc = timed(
        [&](int r) {
            k_probe_reads<<<blocks, PR_THREADS, 0, s>>>(words, (uint64_t)n_words, rounds, 12345u + 7919u * r, sink);
        },
        repeats, s, ms_out);
    cudaFree(sink);
    if (reads_out) *reads_out = (int64_t)blocks * PR_THREADS * rounds * PR_LANES;
    return rc;
}

extern "C" int mp_probe_fma_rate(int kind, int blocks, int iters, int repeats, void* cuda_stream, float* ms_out,
                                 double* flops_out) {
    if (kind < 0 || kind > 2 || blocks < 1 || iters < 1 || repeats < 1 || !ms_out) return MP_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess) return MP_ECUDA;
    int rc;
    if (kind == 0)
        rc = timed([&](int) { k_probe_fma<float><<<blocks, PR_THREADS, 0, s>>>(iters, 0.999f, 1e-3f, (float*)sink); },
                   repeats, s, ms_out);
    else if (kind == 1)
        rc = timed([&](int) { k_probe_fma2<<<blocks, PR_THREADS, 0, s>>>(iters, 0.999f, 1e-3f, (float*)sink); },
                   repeats, s, ms_out);
    else
        rc = timed([&](int) { k_probe_fma<double><<<blocks, PR_THREADS, 0, s>>>(iters, 0.999, 1e-3, sink); },
                   repeats, s, ms_out);
    cudaFree(sink);
    if (flops_out) *flops_out = 2.0 * 16.0 * (double)iters * (double)blocks * PR_THREADS;
    return rc;
}
