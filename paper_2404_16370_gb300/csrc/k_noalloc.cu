// Allocation-free variant of the initial-posterior normalisation.
//
// Some callers of this library cannot allocate device memory at the point
// where they need the posterior: a real-time control loop that does all of
// its allocation at start-up (cudaMalloc may synchronise the device and take
// milliseconds), a host application whose device memory is owned by another
// allocator or budget, or code that runs between a pre-allocation phase and a
// latency-critical phase. mp_posterior_init_noalloc serves them: it takes the
// caller's input and output buffers and keeps its block partials in the
// file-scope array below, so it calls no cudaMalloc, cudaFree or allocating
// library routine.
//
// The array is a fixed MP_NOALLOC_SCRATCH_BYTES held by every device that
// loads this library until the process exits. Every call shares it: calls that
// overlap on the GPU (two streams, or two threads) race on it and must be
// serialised by the caller. Nothing in it carries over between calls: each
// partial slot a call reads is written earlier in the same call.
//
// With lazy module loading (the CUDA default) the first call on a device also
// loads this file's module there, which places the array and the kernels'
// code on the device: that first call is a warm-up for the caller's
// allocation phase, not for its latency-critical phase.
#include "mp_internal.cuh"

#include <cfloat>
#include <climits>
#include <mutex>

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_ITEMS = 8;                       // elements per thread
constexpr int NA_TILE = NA_THREADS * NA_ITEMS;    // elements per block
constexpr int64_t NA_MAX_N = MP_NOALLOC_MAX_PARTICLES;
constexpr int NA_MAX_BLOCKS = (int)((NA_MAX_N + NA_TILE - 1) / NA_TILE);

// layout of the scratch array: four per-block partial arrays, then scalars
struct NaScratch {
    double part_max[NA_MAX_BLOCKS];
    double part_sum[NA_MAX_BLOCKS];
    double part_val[NA_MAX_BLOCKS];
    long long part_idx[NA_MAX_BLOCKS];
    double gmax, gsum;
};

}  // namespace

static __device__ __align__(256) unsigned char mp_noalloc_scratch[MP_NOALLOC_SCRATCH_BYTES];

namespace {

static_assert(sizeof(NaScratch) <= MP_NOALLOC_SCRATCH_BYTES, "scratch array too small");

__device__ __forceinline__ double na_l(const double* lp, const float* ll, int64_t i) {
    return (lp ? lp[i] : 0.0) + (double)ll[i];
}

__device__ __forceinline__ void na_argmax(double& v, long long& i, double v2, long long i2) {
    if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

// block maxima of l = log prior + log-likelihood
__global__ void __launch_bounds__(NA_THREADS) k_na_max(const double* __restrict__ lp, const float* __restrict__ ll,
                                                       int64_t n, NaScratch* S) {
    __shared__ double sm[NA_THREADS / 32];
    double m = -INFINITY;
    int64_t base = (int64_t)blockIdx.x * NA_TILE + threadIdx.x;
#pragma unroll
    for (int k = 0; k < NA_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * NA_THREADS;
        if (i < n) m = fmax(m, na_l(lp, ll, i));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = -INFINITY;
        for (int w = 0; w < NA_THREADS / 32; ++w) v = fmax(v, sm[w]);
        S->part_max[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(1024) k_na_max_final(int nb, NaScratch* S) {
    __shared__ double sm[32];
    double m = -INFINITY;
    for (int b = threadIdx.x; b < nb; b += 1024) m = fmax(m, S->part_max[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = -INFINITY;
        for (int w = 0; w < 32; ++w) v = fmax(v, sm[w]);
        S->gmax = v;
    }
}

// p = exp(l - max l) (unnormalised, into the output), block sums and argmax
__global__ void __launch_bounds__(NA_THREADS) k_na_exp(const double* __restrict__ lp, const float* __restrict__ ll,
                                                       int64_t n, double* __restrict__ post, NaScratch* S) {
    __shared__ double ss[NA_THREADS / 32], sv[NA_THREADS / 32];
    __shared__ long long si[NA_THREADS / 32];
    const double gmax = S->gmax;
    double s = 0.0, bv = -INFINITY;
    long long bi = LLONG_MAX;
    int64_t base = (int64_t)blockIdx.x * NA_TILE + threadIdx.x;
#pragma unroll
    for (int k = 0; k < NA_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * NA_THREADS;
        if (i < n) {
            double v = exp(na_l(lp, ll, i) - gmax);
            post[i] = v;
            s += v;
            na_argmax(bv, bi, v, (long long)i);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        long long i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        na_argmax(bv, bi, v2, i2);
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sv[threadIdx.x >> 5] = bv;
        si[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S0 = 0.0, V = -INFINITY;
        long long I = LLONG_MAX;
        for (int w = 0; w < NA_THREADS / 32; ++w) {
            S0 += ss[w];
            na_argmax(V, I, sv[w], si[w]);
        }
        S->part_sum[blockIdx.x] = S0;
        S->part_val[blockIdx.x] = V;
        S->part_idx[blockIdx.x] = I;
    }
}

__global__ void __launch_bounds__(1024) k_na_final(int nb, NaScratch* S, int64_t* __restrict__ best) {
    __shared__ double ss[32], sv[32];
    __shared__ long long si[32];
    double s = 0.0, bv = -INFINITY;
    long long bi = LLONG_MAX;
    for (int b = threadIdx.x; b < nb; b += 1024) {
        s += S->part_sum[b];
        na_argmax(bv, bi, S->part_val[b], S->part_idx[b]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        long long i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        na_argmax(bv, bi, v2, i2);
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sv[threadIdx.x >> 5] = bv;
        si[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S0 = 0.0, V = -INFINITY;
        long long I = LLONG_MAX;
        for (int w = 0; w < 32; ++w) {
            S0 += ss[w];
            na_argmax(V, I, sv[w], si[w]);
        }
        // Degenerate input: every l_i = -inf, or some l_i NaN or +inf. The
        // normaliser is then not a finite positive number; the outputs get the
        // sentinels best = -1 and post = NaN (x / NaN) instead of an index
        // that no particle has.
        const bool ok = S0 > 0.0 && S0 <= DBL_MAX && I != LLONG_MAX;
        S->gsum = ok ? S0 : __longlong_as_double(0x7ff8000000000000LL);
        *best = ok ? (int64_t)I : (int64_t)-1;
    }
}

__global__ void k_na_normalise(int64_t n, double* __restrict__ post, const NaScratch* S) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) post[i] = post[i] / S->gsum;
}

// Device address of the scratch array, looked up once per device (with that
// device current) and cached.
std::mutex g_na_mutex;
void* g_na_addr[64];
bool g_na_ready[64];

// The kernels dereference every pointer they are given as device memory of
// the current device. A host array (pageable or pinned), or memory of another
// device, is refused before any launch (cudaPointerGetAttributes allocates
// nothing).
int na_check_ptr(const void* p, int dev, const char* name) {
    cudaPointerAttributes a;
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();   // the failed query leaves a (non-sticky) error behind: clear it
        return mp_fail_noctx(MP_EINVAL, "mp_posterior_init_noalloc: %s is not a device pointer", name);
    }
    if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != dev)
        return mp_fail_noctx(MP_EINVAL, "mp_posterior_init_noalloc: %s is not device memory of the current device %d",
                             name, dev);
    return MP_OK;
}

}  // namespace

extern "C" int mp_posterior_init_noalloc(const double* log_prior, const float* loglik, int64_t n, double* post_out,
                                         int64_t* best_out, void* cuda_stream) {
    if (!loglik || !post_out || !best_out)
        return mp_fail_noctx(MP_EINVAL, "mp_posterior_init_noalloc: NULL loglik, post_out or best_out");
    if (n <= 0 || n > NA_MAX_N)
        return mp_fail_noctx(MP_EINVAL, "mp_posterior_init_noalloc: n = %lld outside [1, %lld] (the fixed scratch "
                                        "holds %d block partials)", (long long)n, (long long)NA_MAX_N, NA_MAX_BLOCKS);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64)
        return mp_fail_noctx(MP_ECUDA, "mp_posterior_init_noalloc: no current CUDA device");
    int rc;
    if ((log_prior && (rc = na_check_ptr(log_prior, dev, "log_prior"))) ||
        (rc = na_check_ptr(loglik, dev, "loglik")) || (rc = na_check_ptr(post_out, dev, "post_out")) ||
        (rc = na_check_ptr(best_out, dev, "best_out")))
        return rc;
    NaScratch* S = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_ready[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, mp_noalloc_scratch);
            if (e != cudaSuccess || !ptr)
                return mp_fail_noctx(MP_ECUDA, "mp_posterior_init_noalloc: scratch lookup: %s", cudaGetErrorString(e));
            g_na_addr[dev] = ptr;
            g_na_ready[dev] = true;
        }
        S = (NaScratch*)g_na_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int nb = (int)((n + NA_TILE - 1) / NA_TILE);
    k_na_max<<<nb, NA_THREADS, 0, st>>>(log_prior, loglik, n, S);
    k_na_max_final<<<1, 1024, 0, st>>>(nb, S);
    k_na_exp<<<nb, NA_THREADS, 0, st>>>(log_prior, loglik, n, post_out, S);
    k_na_final<<<1, 1024, 0, st>>>(nb, S, best_out);
    k_na_normalise<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, post_out, S);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return mp_fail_noctx(MP_ECUDA, "mp_posterior_init_noalloc: launch: %s", cudaGetErrorString(e));
    return MP_OK;
}
