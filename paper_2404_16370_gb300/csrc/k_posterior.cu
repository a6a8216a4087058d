// Posterior propagation on the neighbour-particle graph (Sec. III-D, Eq. 11)
// and the representative state:
//   l_i = log prior_i + log p(P | x_i); p_i = exp(l_i - max l) (FP64);
//   post_iters Jacobi sweeps p'_i = sum_j w_ij p_j over the list of i with
//   w_ij = k_ij / sum_j k_ij fixed for the step (one thread per particle, FP64
//   fused multiply-adds);
//   normalise; best = argmax (smallest index on ties); log prior <- log p'.
// Grid-wide max / sum / argmax are two-level (block partials, one final
// block), so results do not depend on atomics' order.
#include "mp_internal.cuh"

namespace {

constexpr int PB = 256;

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ void argmax_merge(double& v, int64_t& i, double v2, int64_t i2) {
    if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

__global__ void __launch_bounds__(PB) k_post_l(const double* __restrict__ logprior, const float* __restrict__ loglik,
                                               int64_t n, double* __restrict__ lbuf, double* __restrict__ part) {
    __shared__ double s[PB / 32];
    int64_t i = blockIdx.x * (int64_t)PB + threadIdx.x;
    double l = -INFINITY;
    if (i < n) {
        l = logprior[i] + (double)loglik[i];
        lbuf[i] = l;
    }
    l = warp_max(l);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < PB / 32 ? s[threadIdx.x] : -INFINITY;
        v = warp_max(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(1024) k_reduce_max(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double s[32];
    double v = -INFINITY;
    for (int k = threadIdx.x; k < nb; k += 1024) v = fmax(v, part[k]);
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = s[threadIdx.x];
        v = warp_max(v);
        if (threadIdx.x == 0) *out = v;
    }
}

__global__ void __launch_bounds__(PB) k_post_exp(const double* __restrict__ lbuf, int64_t n,
                                                 const double* __restrict__ mx, double* __restrict__ p0,
                                                 double* __restrict__ p, double* __restrict__ part) {
    __shared__ double s[PB / 32];
    int64_t i = blockIdx.x * (int64_t)PB + threadIdx.x;
    double v = 0.0;
    if (i < n) {
        v = exp(lbuf[i] - *mx);
        p0[i] = v;
        p[i] = v;
    }
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < PB / 32 ? s[threadIdx.x] : 0.0;
        w = warp_sum(w);
        if (threadIdx.x == 0) part[blockIdx.x] = w;
    }
}

__global__ void __launch_bounds__(1024) k_reduce_sum(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double s[32];
    double v = 0.0;
    for (int k = threadIdx.x; k < nb; k += 1024) v += part[k];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = s[threadIdx.x];
        v = warp_sum(v);
        if (threadIdx.x == 0) *out = v;
    }
}

// Normalised weights w_ij = k_ij / sum_j k_ij (FP64) and 1 / sum_j k_ij,
// fixed for the sweeps of a step: a sweep entry is then one FP64 fused
// multiply-add (GB300's FP64 rate is low, so the division and the FP32 -> FP64
// conversion are taken out of the ten sweeps).
__global__ void k_post_weights(int64_t n, int K, const int32_t* __restrict__ ids, const float* __restrict__ kk,
                               double* __restrict__ w, double* __restrict__ inv_den) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double den = 0.0;
    for (int l = 0; l < K; ++l)
        if (ids[i * K + l] >= 0) den += (double)kk[i * K + l];
    const double inv = den > 0.0 ? 1.0 / den : 0.0;
    for (int l = 0; l < K; ++l) w[i * K + l] = ids[i * K + l] >= 0 ? (double)kk[i * K + l] * inv : 0.0;
    inv_den[i] = inv;
}

// One Jacobi sweep of Eq. 11, one thread per particle: p'_i = sum_j w_ij p_j
// with FP64 fused multiply-adds over the list (rows read with 16-byte loads
// when the list length is a multiple of 4); a particle whose kernel weights
// sum to zero keeps its value.
template <int KT>
__global__ void __launch_bounds__(256) k_post_sweep(const double* __restrict__ pin, double* __restrict__ pout, int64_t n,
                                                    int Krt, const int32_t* __restrict__ ids,
                                                    const double* __restrict__ w, const double* __restrict__ inv_den) {
    const int K = KT > 0 ? KT : Krt;   // compile-time list length for the common sizes
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double num = 0.0;
    if (KT > 0 && KT % 4 == 0) {
        const int4* row = reinterpret_cast<const int4*>(ids + i * KT);
        const double2* wr = reinterpret_cast<const double2*>(w + i * KT);
#pragma unroll
        for (int q = 0; q < KT / 4; ++q) {
            const int4 j4 = __ldg(row + q);
            const double2 w0 = __ldg(wr + 2 * q), w1 = __ldg(wr + 2 * q + 1);
            if (j4.x >= 0 && MP_DCHECK(j4.x < n, "neighbour id", j4.x)) num = fma(w0.x, __ldg(pin + j4.x), num);
            if (j4.y >= 0 && MP_DCHECK(j4.y < n, "neighbour id", j4.y)) num = fma(w0.y, __ldg(pin + j4.y), num);
            if (j4.z >= 0 && MP_DCHECK(j4.z < n, "neighbour id", j4.z)) num = fma(w1.x, __ldg(pin + j4.z), num);
            if (j4.w >= 0 && MP_DCHECK(j4.w < n, "neighbour id", j4.w)) num = fma(w1.y, __ldg(pin + j4.w), num);
        }
    } else {
        for (int l = 0; l < K; ++l) {
            const int j = __ldg(ids + i * K + l);
            if (j >= 0 && MP_DCHECK(j < n, "neighbour id", j)) num = fma(__ldg(w + i * K + l), __ldg(pin + j), num);
        }
    }
    pout[i] = inv_den[i] > 0.0 ? num : pin[i];
}

__global__ void __launch_bounds__(PB) k_post_final_part(const double* __restrict__ p, int64_t n,
                                                        double* __restrict__ part_sum, double* __restrict__ part_max,
                                                        int64_t* __restrict__ part_idx) {
    __shared__ double ss[PB / 32], sm[PB / 32];
    __shared__ int64_t si[PB / 32];
    int64_t i = blockIdx.x * (int64_t)PB + threadIdx.x;
    double v = i < n ? p[i] : 0.0;
    double m = i < n ? v : -INFINITY;
    int64_t mi = i < n ? i : INT64_MAX;
    double s = warp_sum(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double m2 = __shfl_xor_sync(0xffffffffu, m, o);
        int64_t i2 = __shfl_xor_sync(0xffffffffu, mi, o);
        argmax_merge(m, mi, m2, i2);
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sm[threadIdx.x >> 5] = m;
        si[threadIdx.x >> 5] = mi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, M = -INFINITY;
        int64_t I = INT64_MAX;
        for (int k = 0; k < PB / 32; ++k) {
            S += ss[k];
            argmax_merge(M, I, sm[k], si[k]);
        }
        part_sum[blockIdx.x] = S;
        part_max[blockIdx.x] = M;
        part_idx[blockIdx.x] = I;
    }
}

__global__ void __launch_bounds__(1024) k_post_final_reduce(const double* __restrict__ part_sum,
                                                            const double* __restrict__ part_max,
                                                            const int64_t* __restrict__ part_idx, int nb,
                                                            double* __restrict__ scalars, int64_t* __restrict__ best) {
    __shared__ double ss[32], sm[32];
    __shared__ int64_t si[32];
    double S = 0.0, M = -INFINITY;
    int64_t I = INT64_MAX;
    for (int k = threadIdx.x; k < nb; k += 1024) {
        S += part_sum[k];
        argmax_merge(M, I, part_max[k], part_idx[k]);
    }
    S = warp_sum(S);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double m2 = __shfl_xor_sync(0xffffffffu, M, o);
        int64_t i2 = __shfl_xor_sync(0xffffffffu, I, o);
        argmax_merge(M, I, m2, i2);
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = S;
        sm[threadIdx.x >> 5] = M;
        si[threadIdx.x >> 5] = I;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S2 = 0.0, M2 = -INFINITY;
        int64_t I2 = INT64_MAX;
        for (int k = 0; k < 32; ++k) {
            S2 += ss[k];
            argmax_merge(M2, I2, sm[k], si[k]);
        }
        scalars[2] = S2;
        scalars[3] = M2 / S2;
        *best = I2;
    }
}

__global__ void k_post_normalise(const double* __restrict__ p, int64_t n, const double* __restrict__ scalars,
                                 const int64_t* __restrict__ best, const float4* __restrict__ poses,
                                 double* __restrict__ post, double* __restrict__ logprior, float4* __restrict__ best_pose) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = p[i] / scalars[2];
    post[i] = v;
    logprior[i] = log(v);
    if (i == *best) {
        best_pose[0] = poses[2 * i];
        best_pose[1] = poses[2 * i + 1];
    }
}

template <int KT>
int sweeps(mp_ctx* c, double*& a, double*& b, const double* inv_den) {
    for (int it = 0; it < c->p.post_iters; ++it) {
        k_post_sweep<KT><<<grid_for(c->n, 256), 256, 0, c->stream>>>(a, b, c->n, c->p.K, c->nbr_ids[c->nbr_cur],
                                                                    c->post_w, inv_den);
        MP_LAUNCHED(c);
        double* t = a;
        a = b;
        b = t;
    }
    return MP_OK;
}



}  // namespace

int mp_launch_posterior(mp_ctx* c) {
    int64_t n = c->n;
    int nb = (int)((n + PB - 1) / PB);
    double* part = c->red;
    double* part2 = c->red + nb;
    int64_t* part_idx = (int64_t*)(c->red + 2 * (int64_t)nb);
    double* lbuf = c->post;   // scratch until the final normalisation
    k_post_l<<<nb, PB, 0, c->stream>>>(c->logprior, c->loglik, n, lbuf, part);
    MP_LAUNCHED(c);
    k_reduce_max<<<1, 1024, 0, c->stream>>>(part, nb, &c->scalars[0]);
    MP_LAUNCHED(c);
    k_post_exp<<<nb, PB, 0, c->stream>>>(lbuf, n, &c->scalars[0], c->post_init, c->post_tmp, part);
    MP_LAUNCHED(c);
    k_reduce_sum<<<1, 1024, 0, c->stream>>>(part, nb, &c->scalars[1]);
    MP_LAUNCHED(c);
    k_post_weights<<<grid_for(n, 256), 256, 0, c->stream>>>(n, c->p.K, c->nbr_ids[c->nbr_cur], c->nbr_k, c->post_w,
                                                            c->post_invden);
    MP_LAUNCHED(c);
    double* a = c->post_tmp;
    double* b = c->post;
    int rc;
    if (c->p.K == 32) rc = sweeps<32>(c, a, b, c->post_invden);
    else if (c->p.K == 16) rc = sweeps<16>(c, a, b, c->post_invden);
    else rc = sweeps<0>(c, a, b, c->post_invden);
    if (rc) return rc;
    // a holds the smoothed (unnormalised) posterior
    k_post_final_part<<<nb, PB, 0, c->stream>>>(a, n, part, part2, part_idx);
    MP_LAUNCHED(c);
    k_post_final_reduce<<<1, 1024, 0, c->stream>>>(part, part2, part_idx, nb, c->scalars, c->best_idx);
    MP_LAUNCHED(c);
    double* dst = c->post;
    if (a == c->post) {
        // normalise out of post_tmp's twin: copy a first so that post can be written
        MP_CUDA(c, cudaMemcpyAsync(c->post_tmp, a, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
        a = c->post_tmp;
    }
    k_post_normalise<<<grid_for(n, 256), 256, 0, c->stream>>>(a, n, c->scalars, c->best_idx, c->poses[c->cur], dst,
                                                              c->logprior, c->best_pose);
    MP_LAUNCHED(c);
    return MP_OK;
}
