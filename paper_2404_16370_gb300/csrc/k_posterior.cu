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

// One instance's posterior stage. post doubles as the buffer of l until the
// normalisation; the sweeps alternate post_tmp -> post -> post_tmp ...
struct PostArgs {
    const float* loglik;
    double* logprior;
    int64_t n;
    int nb;               // blocks of PB particles
    double* post;
    double* post_tmp;
    double* post_init;
    double* part;         // nb block partials (max, then sums)
    double* part2;        // nb block maxima of the final pass
    int64_t* part_idx;    // nb block argmaxes
    double* scalars;      // [0] max l, [1] sum exp, [2] sum post, [3] best prob
    int64_t* best_idx;
    const int32_t* ids;
    int K;
    const float* kk;
    double* w;            // normalised weights, slot-major: w[l * n + i]
    int32_t* ids_t;       // the ids, slot-major: ids_t[l * n + i]
    double* invden;       // 1 / sum_j k_ij
    int iters;
    const float4* poses;
    float4* best_pose;
};

struct PostLOp {
    using Args = PostArgs;
    static constexpr int THREADS = PB, MINB = 1;
    static __device__ __forceinline__ void run(const PostArgs& A, unsigned bx, unsigned) {
        __shared__ double s[PB / 32];
        int64_t i = (int64_t)bx * PB + threadIdx.x;
        double l = -INFINITY;
        if (i < A.n) {
            l = A.logprior[i] + (double)A.loglik[i];
            A.post[i] = l;
        }
        l = warp_max(l);
        if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = l;
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < PB / 32 ? s[threadIdx.x] : -INFINITY;
            v = warp_max(v);
            if (threadIdx.x == 0) A.part[bx] = v;
        }
    }
};

struct ReduceMaxOp {
    using Args = PostArgs;
    static constexpr int THREADS = 1024, MINB = 1;
    static __device__ __forceinline__ void run(const PostArgs& A, unsigned, unsigned) {
        __shared__ double s[32];
        double v = -INFINITY;
        for (int k = threadIdx.x; k < A.nb; k += 1024) v = fmax(v, A.part[k]);
        v = warp_max(v);
        if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            v = s[threadIdx.x];
            v = warp_max(v);
            if (threadIdx.x == 0) A.scalars[0] = v;
        }
    }
};

struct PostExpOp {
    using Args = PostArgs;
    static constexpr int THREADS = PB, MINB = 1;
    static __device__ __forceinline__ void run(const PostArgs& A, unsigned bx, unsigned) {
        __shared__ double s[PB / 32];
        int64_t i = (int64_t)bx * PB + threadIdx.x;
        double v = 0.0;
        if (i < A.n) {
            v = exp(A.post[i] - A.scalars[0]);
            A.post_init[i] = v;
            A.post_tmp[i] = v;
        }
        v = warp_sum(v);
        if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            double w = threadIdx.x < PB / 32 ? s[threadIdx.x] : 0.0;
            w = warp_sum(w);
            if (threadIdx.x == 0) A.part[bx] = w;
        }
    }
};

struct ReduceSumOp {
    using Args = PostArgs;
    static constexpr int THREADS = 1024, MINB = 1;
    static __device__ __forceinline__ void run(const PostArgs& A, unsigned, unsigned) {
        __shared__ double s[32];
        double v = 0.0;
        for (int k = threadIdx.x; k < A.nb; k += 1024) v += A.part[k];
        v = warp_sum(v);
        if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            v = s[threadIdx.x];
            v = warp_sum(v);
            if (threadIdx.x == 0) A.scalars[1] = v;
        }
    }
};

// Normalised weights w_ij = k_ij / sum_j k_ij (FP64) and 1 / sum_j k_ij,
// fixed for the sweeps of a step: a sweep entry is then one FP64 fused
// multiply-add (GB300's FP64 rate is low, so the division and the FP32 -> FP64
// conversion are taken out of the ten sweeps). Weights and ids are written
// slot-major ([l * n + i]) so that the sweeps' loads are coalesced.
struct PostWeightsOp {
    using Args = PostArgs;
    static constexpr int THREADS = 256, MINB = 1;
    static __device__ __forceinline__ void run(const PostArgs& A, unsigned bx, unsigned) {
        const int64_t n = A.n;
        const int K = A.K;
        const int32_t* __restrict__ ids = A.ids;
        const float* __restrict__ kk = A.kk;
        double* __restrict__ w = A.w;
        int64_t i = (int64_t)bx * THREADS + threadIdx.x;
        if (i >= n) return;
        double den = 0.0;
        for (int l = 0; l < K; ++l)
            if (ids[i * K + l] >= 0) den += (double)kk[i * K + l];
        const double inv = den > 0.0 ? 1.0 / den : 0.0;
        for (int l = 0; l < K; ++l) {
            const int32_t j = ids[i * K + l];
            w[l * n + i] = j >= 0 ? (double)kk[i * K + l] * inv : 0.0;
            A.ids_t[l * n + i] = j;
        }
        A.invden[i] = inv;
    }
};

// Jacobi sweep `it` (the block map's y index) of Eq. 11, one thread per
// particle: p'_i = sum_j w_ij p_j with FP64 fused multiply-adds over the list
// in slot order (slot-major ids and weights: a warp's loads of one slot are
// contiguous); a particle whose kernel weights sum to zero keeps its value.
template <int KT>
struct PostSweepOp {
    using Args = PostArgs;
    static constexpr int THREADS = 256, MINB = 1;
    static __device__ __forceinline__ void run(const PostArgs& A, unsigned bx, unsigned it) {
        const double* __restrict__ pin = (it & 1) ? A.post : A.post_tmp;
        double* __restrict__ pout = (it & 1) ? A.post_tmp : A.post;
        const int64_t n = A.n;
        const int32_t* __restrict__ ids = A.ids_t;
        const double* __restrict__ w = A.w;
        const int K = KT > 0 ? KT : A.K;   // compile-time list length for the common sizes
        int64_t i = (int64_t)bx * THREADS + threadIdx.x;
        if (i >= n) return;
        double num = 0.0;
#pragma unroll(KT > 0 ? KT : 1)
        for (int l = 0; l < K; ++l) {
            const int j = __ldg(ids + l * n + i);
            if (j >= 0 && MP_DCHECK(j < n, "neighbour id", j)) num = fma(__ldg(w + l * n + i), __ldg(pin + j), num);
        }
        pout[i] = A.invden[i] > 0.0 ? num : pin[i];
    }
};

// the smoothed posterior after the sweeps
__device__ __forceinline__ const double* post_smoothed(const PostArgs& A) { return (A.iters & 1) ? A.post : A.post_tmp; }

struct FinalPartOp {
    using Args = PostArgs;
    static constexpr int THREADS = PB, MINB = 1;
    static __device__ __forceinline__ void run(const PostArgs& A, unsigned bx, unsigned) {
        __shared__ double ss[PB / 32], sm[PB / 32];
        __shared__ int64_t si[PB / 32];
        const double* __restrict__ p = post_smoothed(A);
        int64_t i = (int64_t)bx * PB + threadIdx.x;
        double v = i < A.n ? p[i] : 0.0;
        double m = i < A.n ? v : -INFINITY;
        int64_t mi = i < A.n ? i : INT64_MAX;
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
            A.part[bx] = S;
            A.part2[bx] = M;
            A.part_idx[bx] = I;
        }
    }
};

struct FinalReduceOp {
    using Args = PostArgs;
    static constexpr int THREADS = 1024, MINB = 1;
    static __device__ __forceinline__ void run(const PostArgs& A, unsigned, unsigned) {
        __shared__ double ss[32], sm[32];
        __shared__ int64_t si[32];
        double S = 0.0, M = -INFINITY;
        int64_t I = INT64_MAX;
        for (int k = threadIdx.x; k < A.nb; k += 1024) {
            S += A.part[k];
            argmax_merge(M, I, A.part2[k], A.part_idx[k]);
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
            A.scalars[2] = S2;
            A.scalars[3] = M2 / S2;
            *A.best_idx = I2;
        }
    }
};

// normalise out of post_tmp (after an odd number of sweeps the smoothed values
// are copied there first), store the log prior, copy the best pose
struct NormaliseOp {
    using Args = PostArgs;
    static constexpr int THREADS = 256, MINB = 1;
    static __device__ __forceinline__ void run(const PostArgs& A, unsigned bx, unsigned) {
        int64_t i = (int64_t)bx * THREADS + threadIdx.x;
        if (i >= A.n) return;
        double v = A.post_tmp[i] / A.scalars[2];
        A.post[i] = v;
        A.logprior[i] = log(v);
        if (i == *A.best_idx) {
            A.best_pose[0] = A.poses[2 * i];
            A.best_pose[1] = A.poses[2 * i + 1];
        }
    }
};

template <typename Op>
__global__ void __launch_bounds__(Op::THREADS) k_post(const PostArgs A, int y) {
    Op::run(A, blockIdx.x, y);
}

PostArgs post_args(mp_ctx* c, int cur) {
    PostArgs A;
    A.loglik = c->loglik;
    A.logprior = c->logprior;
    A.n = c->n;
    A.nb = (int)((c->n + PB - 1) / PB);
    A.post = c->post;
    A.post_tmp = c->post_tmp;
    A.post_init = c->post_init;
    A.part = c->red;
    A.part2 = c->red + A.nb;
    A.part_idx = (int64_t*)(c->red + 2 * (int64_t)A.nb);
    A.scalars = c->scalars;
    A.best_idx = c->best_idx;
    A.ids = c->nbr_ids[cur];
    A.K = c->p.K;
    A.kk = c->nbr_k;
    A.w = c->post_w;
    A.ids_t = c->post_ids;
    A.invden = c->post_invden;
    A.iters = c->p.post_iters;
    A.poses = c->poses[c->cur];
    A.best_pose = c->best_pose;
    return A;
}

template <int KT>
void sweeps(mp_ctx* c, const PostArgs& A) {
    for (int it = 0; it < A.iters; ++it) k_post<PostSweepOp<KT>><<<grid_for(A.n, 256), 256, 0, c->stream>>>(A, it);
}

}  // namespace

int mp_launch_posterior(mp_ctx* c) {
    const PostArgs A = post_args(c, c->nbr_cur);
    const unsigned nb = (unsigned)A.nb;
    k_post<PostLOp><<<nb, PB, 0, c->stream>>>(A, 0);
    MP_LAUNCHED(c);
    k_post<ReduceMaxOp><<<1, 1024, 0, c->stream>>>(A, 0);
    MP_LAUNCHED(c);
    k_post<PostExpOp><<<nb, PB, 0, c->stream>>>(A, 0);
    MP_LAUNCHED(c);
    k_post<ReduceSumOp><<<1, 1024, 0, c->stream>>>(A, 0);
    MP_LAUNCHED(c);
    k_post<PostWeightsOp><<<grid_for(A.n, 256), 256, 0, c->stream>>>(A, 0);
    MP_LAUNCHED(c);
    if (A.K == 32) sweeps<32>(c, A);
    else if (A.K == 16) sweeps<16>(c, A);
    else sweeps<0>(c, A);
    c->launches += A.iters - 1;
    MP_LAUNCHED(c);
    k_post<FinalPartOp><<<nb, PB, 0, c->stream>>>(A, 0);
    MP_LAUNCHED(c);
    k_post<FinalReduceOp><<<1, 1024, 0, c->stream>>>(A, 0);
    MP_LAUNCHED(c);
    if (A.iters & 1)
        MP_CUDA(c, cudaMemcpyAsync(c->post_tmp, c->post, sizeof(double) * (size_t)A.n, cudaMemcpyDeviceToDevice,
                                   c->stream));
    k_post<NormaliseOp><<<grid_for(A.n, 256), 256, 0, c->stream>>>(A, 0);
    MP_LAUNCHED(c);
    return MP_OK;
}

// Grouped posterior: the same launches over all instances; the sweeps of
// instances with K = 32, 16 and other list lengths go in separate launches.
int mp_plan_posterior(mp_group* G, int p, std::vector<GOp>& plan) {
    std::vector<PostArgs> tab;
    std::vector<int64_t> bpb, b1;
    std::vector<int> odd;
    int max_iters = 0;
    for (int i = 0; i < G->size(); ++i) {
        mp_ctx* c = G->ctx[i];
        tab.push_back(post_args(c, c->nbr_cur ^ p ^ 1));   // the list the merge of this step wrote
        bpb.push_back(tab.back().nb);
        b1.push_back(1);
        max_iters = tab.back().iters > max_iters ? tab.back().iters : max_iters;
        if (tab.back().iters & 1) odd.push_back(i);
    }
    const PostArgs* t = G->upload(tab);
    unsigned npb = 0, n1 = 0;
    const GBlk* mpb = G->block_map(bpb, &npb);
    const GBlk* m1 = G->block_map(b1, &n1);
    plan_kernel<PostLOp>(plan, t, mpb, npb);
    plan_kernel<ReduceMaxOp>(plan, t, m1, n1);
    plan_kernel<PostExpOp>(plan, t, mpb, npb);
    plan_kernel<ReduceSumOp>(plan, t, m1, n1);
    plan_kernel<PostWeightsOp>(plan, t, mpb, npb);   // PB = 256 threads: the same blocks
    for (int it = 0; it < max_iters; ++it) {
        std::vector<GBlk> m32, m16, m0;
        for (int i = 0; i < G->size(); ++i) {
            if (tab[i].iters <= it) continue;
            std::vector<GBlk>& m = tab[i].K == 32 ? m32 : tab[i].K == 16 ? m16 : m0;
            for (int64_t b = 0; b < bpb[i]; ++b) m.push_back(GBlk{i, (int32_t)b, it, 0});
        }
        if (!m32.empty()) plan_kernel<PostSweepOp<32>>(plan, t, G->upload(m32), (unsigned)m32.size());
        if (!m16.empty()) plan_kernel<PostSweepOp<16>>(plan, t, G->upload(m16), (unsigned)m16.size());
        if (!m0.empty()) plan_kernel<PostSweepOp<0>>(plan, t, G->upload(m0), (unsigned)m0.size());
    }
    plan_kernel<FinalPartOp>(plan, t, mpb, npb);
    plan_kernel<FinalReduceOp>(plan, t, m1, n1);
    for (int i : odd)
        plan_copy(plan, G->ctx[i]->post_tmp, G->ctx[i]->post, sizeof(double) * (size_t)G->ctx[i]->n);
    plan_kernel<NormaliseOp>(plan, t, mpb, npb);
    return G->err;
}
