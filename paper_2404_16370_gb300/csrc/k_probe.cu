// Measurement helper: the rate of independent, uniformly random 4-byte reads
// over a device buffer, a reference for the likelihood's NNF lookups while
// particles are spread (those are random across particles but clustered
// along one particle's scan, so they keep more DRAM rows open).
#include "mp_internal.cuh"

namespace {

__global__ void __launch_bounds__(256) k_probe_reads(const uint32_t* __restrict__ words, uint64_t n_words, int reads,
                                                     uint32_t seed, uint32_t* __restrict__ sink) {
    const uint64_t tid = (uint64_t)blockIdx.x * 256 + threadIdx.x;
    // per-thread LCG state (Numerical Recipes constants), scrambled start
    uint32_t x = (uint32_t)(tid * 2654435761ull) ^ seed;
    uint32_t acc = 0;
#pragma unroll 8
    for (int r = 0; r < reads; ++r) {
        x = x * 1664525u + 1013904223u;
        const uint64_t idx = ((uint64_t)x * n_words) >> 32;   // uniform in [0, n_words)
        acc += __ldg(words + idx);
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;   // keeps the reads live; practically never taken
}

}  // namespace

extern "C" int mp_probe_random_reads(const uint32_t* words, int64_t n_words, int blocks, int reads_per_thread,
                                     int repeats, void* cuda_stream, float* ms_out) {
    if (!words || !ms_out || n_words < 1 || n_words > ((int64_t)1 << 32) || blocks < 1 || reads_per_thread < 1 ||
        repeats < 1)
        return MP_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint32_t* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MP_OK;
    if (cudaMalloc(&sink, sizeof(uint32_t)) != cudaSuccess) return MP_ECUDA;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = MP_ECUDA;
    if (rc == MP_OK) {
        k_probe_reads<<<blocks, 256, 0, s>>>(words, (uint64_t)n_words, reads_per_thread, 12345u, sink);
        cudaEventRecord(e0, s);
        for (int r = 0; r < repeats; ++r)
            k_probe_reads<<<blocks, 256, 0, s>>>(words, (uint64_t)n_words, reads_per_thread, 777u + 31u * r, sink);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = MP_ECUDA;
        float ms = 0.f;
        if (rc == MP_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = MP_ECUDA;
        *ms_out = ms / repeats;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}
