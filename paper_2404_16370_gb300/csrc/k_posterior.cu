// Posterior propagation on the neighbour-particle graph (Sec. III-D, Eq. 11)
// and the representative state:
//   l_i = log prior_i + log p(P | x_i); p_i = exp(l_i - max l) (FP64);
//   post_iters Jacobi sweeps p'_i = sum_j w_ij p_j over the list of i with
//   w_ij = k_ij / sum_j k_ij fixed for the step (one thread per particle, FP64
//   fused multiply-adds);
//   normalise; best = argmax (smallest index on ties); log prior <- log p'.
// Grid-wide max / sum / argmax are two-level (block partials, then one CTA
// per instance), so results do not depend on atomics' order.
//
// The whole stage is one cooperative (persistent) kernel, k_post_phase: its
// CTAs, all resident, take the particle blocks of one instance (a context's
// own launch) or of every instance of a batch in turn, with a bounded grid
// barrier (grid_sync) between the sub-steps: block maxima | per-instance max |
// exp, block sums and sweep weights | per-instance sum and sweep 1 | sweeps
// 2..iters | final block partials | per-instance sum and argmax | normalise.
// A barrier that gives up records MP_ERR_WAIT for every instance and the
// kernel returns. A context's launch and a batch's launch run the same code
// per block and per instance, so they compute the same bits.
#include "mp_internal.cuh"

#include <algorithm>

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
    double lfloor;        // lower bound of l - max l in the initial posterior (-post_floor; -inf: none)
    const float4* poses;
    float4* best_pose;
    int32_t* err;         // error bits (MP_ERR_WAIT when a grid barrier gives up)
};

// block maxima of l = log prior + log likelihood (l kept in post)
__device__ __forceinline__ void post_l(const PostArgs& A, unsigned bx) {
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

// the instance's max l over its block maxima
__device__ __forceinline__ void reduce_max(const PostArgs& A) {
    __shared__ double s[PB / 32];
    double v = -INFINITY;
    for (int k = threadIdx.x; k < A.nb; k += PB) v = fmax(v, A.part[k]);
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < PB / 32 ? s[threadIdx.x] : -INFINITY;
        v = warp_max(v);
        if (threadIdx.x == 0) A.scalars[0] = v;
    }
}

// p = exp(max(l - max l, floor)) into post_init and post_tmp (the sweeps'
// input); block sums
__device__ __forceinline__ void post_exp(const PostArgs& A, unsigned bx) {
    __shared__ double s[PB / 32];
    int64_t i = (int64_t)bx * PB + threadIdx.x;
    double v = 0.0;
    if (i < A.n) {
        v = exp(fmax(A.post[i] - A.scalars[0], A.lfloor));
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

// the instance's sum of exp(l - max l)
__device__ __forceinline__ void reduce_sum(const PostArgs& A) {
    __shared__ double s[PB / 32];
    double v = 0.0;
    for (int k = threadIdx.x; k < A.nb; k += PB) v += A.part[k];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < PB / 32 ? s[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) A.scalars[1] = v;
    }
}

// Normalised weights w_ij = k_ij / sum_j k_ij (FP64) and 1 / sum_j k_ij,
// fixed for the sweeps of a step: a sweep entry is then one FP64 fused
// multiply-add (GB300's FP64 rate is low, so the division and the FP32 -> FP64
// conversion are taken out of the ten sweeps). Weights and ids are written
// slot-major ([l * n + i]) so that the sweeps' loads are coalesced. The lists
// (row-major, K per particle) pass through shared memory in tiles of WT
// particles: coalesced row loads, a per-particle sum in slot order, coalesced
// slot-major stores.
constexpr int WT = 32;
__device__ __forceinline__ void post_weights(const PostArgs& A, unsigned bx) {
    __shared__ int32_t s_id[WT * (MP_MAXK + 1)];   // row stride K + 1: conflict-free column reads
    __shared__ double s_k[WT * (MP_MAXK + 1)];     // k_ij converted to FP64 once
    __shared__ double s_inv[WT];
    const int64_t n = A.n;
    const int K = A.K, R = A.K + 1;
    const int32_t* __restrict__ ids = A.ids;
    const float* __restrict__ kk = A.kk;
    for (int t = 0; t < PB / WT; ++t) {
        const int64_t i0 = (int64_t)bx * PB + t * WT;
        if (i0 >= n) break;   // block-uniform
        const int np = n - i0 < WT ? (int)(n - i0) : WT;
        const int E = np * K;
        for (int e = threadIdx.x; e < E; e += PB) {
            const int pl = e / K, l = e - pl * K;
            s_id[pl * R + l] = ids[i0 * K + e];
            s_k[pl * R + l] = (double)kk[i0 * K + e];
        }
        __syncthreads();
        if (threadIdx.x < np) {
            double den = 0.0;
            for (int l = 0; l < K; ++l)
                if (s_id[threadIdx.x * R + l] >= 0) den += s_k[threadIdx.x * R + l];
            const double inv = den > 0.0 ? 1.0 / den : 0.0;
            s_inv[threadIdx.x] = inv;
            A.invden[i0 + threadIdx.x] = inv;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < WT * K; e += PB) {
            const int l = e / WT, pl = e - l * WT;
            if (pl < np) {
                const int32_t j = s_id[pl * R + l];
                A.w[l * n + i0 + pl] = j >= 0 ? s_k[pl * R + l] * s_inv[pl] : 0.0;
                A.ids_t[l * n + i0 + pl] = j;
            }
        }
        __syncthreads();
    }
}

// Jacobi sweep `it` of Eq. 11, one thread per particle: p'_i = sum_j w_ij p_j
// with FP64 fused multiply-adds over the list in slot order (slot-major ids
// and weights: a warp's loads of one slot are contiguous); a particle whose
// kernel weights sum to zero keeps its value. Ids, weights and p were written
// earlier in the same launch by other CTAs: L2-coherent loads (ld.global.cg,
// not the read-only path), ordered by the grid barrier's fences; the random
// gathers of p do not allocate in L1.
template <int KT>
__device__ __forceinline__ void post_sweep(const PostArgs& A, unsigned bx, int it) {
    const double* pin = (it & 1) ? A.post : A.post_tmp;
    double* pout = (it & 1) ? A.post_tmp : A.post;
    const int64_t n = A.n;
    const int32_t* ids = A.ids_t;
    const double* w = A.w;
    const int K = KT > 0 ? KT : A.K;   // compile-time list length for the common sizes
    int64_t i = (int64_t)bx * PB + threadIdx.x;
    if (i < n) {
        double num = 0.0;
#pragma unroll(KT > 0 ? KT : 1)
        for (int l = 0; l < K; ++l) {
            const int j = __ldcg(ids + l * n + i);
            if (j >= 0 && MP_DCHECK(j < n, "neighbour id", j)) num = fma(__ldcg(w + l * n + i), __ldcg(pin + j), num);
        }
        pout[i] = __ldcg(A.invden + i) > 0.0 ? num : __ldcg(pin + i);
    }
}

// the smoothed posterior after the sweeps
__device__ __forceinline__ const double* post_smoothed(const PostArgs& A) { return (A.iters & 1) ? A.post : A.post_tmp; }

// block partials of the smoothed posterior: sum, max and its index
__device__ __forceinline__ void final_part(const PostArgs& A, unsigned bx) {
    __shared__ double ss[PB / 32], sm[PB / 32];
    __shared__ int64_t si[PB / 32];
    const double* p = post_smoothed(A);
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

// the instance's sum of the smoothed posterior, its best value and index
__device__ __forceinline__ void final_reduce(const PostArgs& A) {
    __shared__ double ss[PB / 32], sm[PB / 32];
    __shared__ int64_t si[PB / 32];
    double S = 0.0, M = -INFINITY;
    int64_t I = INT64_MAX;
    for (int k = threadIdx.x; k < A.nb; k += PB) {
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
        for (int k = 0; k < PB / 32; ++k) {
            S2 += ss[k];
            argmax_merge(M2, I2, sm[k], si[k]);
        }
        A.scalars[2] = S2;
        A.scalars[3] = M2 / S2;
        *A.best_idx = I2;
    }
}

// normalise (post_tmp keeps the smoothed values), store the log prior, copy
// the best pose
__device__ __forceinline__ void normalise(const PostArgs& A, unsigned bx) {
    int64_t i = (int64_t)bx * PB + threadIdx.x;
    if (i < A.n) {
        const double sm = post_smoothed(A)[i];
        if (A.iters & 1) A.post_tmp[i] = sm;
        const double v = sm / A.scalars[2];
        A.post[i] = v;
        A.logprior[i] = log(v);
        if (i == *A.best_idx) {
            A.best_pose[0] = A.poses[2 * i];
            A.best_pose[1] = A.poses[2 * i + 1];
        }
    }
}

// The launch's argument: one instance (tab null; a context's own launch) or a
// table of instances with the list of their particle blocks (a batch).
struct PostPhase {
    PostArgs one;
    const PostArgs* tab;
    const GBlk* blocks;   // (inst, bx) of every particle block; null: blocks 0..one.nb-1 of `one`
    int n_blocks, n_inst, max_iters, starve;
    GridBar* bar;
    long long budget;
};

__device__ __forceinline__ const PostArgs& phase_args(const PostPhase& P, int inst) {
    return P.tab ? P.tab[inst] : P.one;
}
__device__ __forceinline__ const PostArgs& phase_item(const PostPhase& P, int w, unsigned& bx) {
    if (!P.blocks) {
        bx = (unsigned)w;
        return P.one;
    }
    const GBlk g = P.blocks[w];
    bx = (unsigned)g.bx;
    return P.tab[g.inst];
}

// 4 CTAs of 256 threads per SM: 64 registers, no spill (fewer registers and
// more CTAs spill the sub-steps' FP64 values and measured slower)
__global__ void __launch_bounds__(PB, 4) k_post_phase(const __grid_constant__ PostPhase P) {
    // the test knob: the first barrier waits for one CTA more than the grid
    unsigned expect = gridDim.x + (P.starve ? 1u : 0u);
    auto sync = [&]() {
        const bool ok = grid_sync(P.bar, expect, P.budget);
        expect = gridDim.x;
        if (!ok && threadIdx.x == 0)
            for (int k = 0; k < P.n_inst; ++k) atomicOr(phase_args(P, k).err, MP_ERR_WAIT);
        return ok;
    };
    unsigned bx;
    for (int w = blockIdx.x; w < P.n_blocks; w += gridDim.x) {
        const PostArgs& A = phase_item(P, w, bx);   // sets bx: a statement of its own
        post_l(A, bx);
        __syncthreads();
    }
    if (!sync()) return;
    for (int k = blockIdx.x; k < P.n_inst; k += gridDim.x) {
        reduce_max(phase_args(P, k));
        __syncthreads();
    }
    if (!sync()) return;
    for (int w = blockIdx.x; w < P.n_blocks; w += gridDim.x) {
        const PostArgs& A = phase_item(P, w, bx);
        post_exp(A, bx);
        post_weights(A, bx);
        __syncthreads();
    }
    if (!sync()) return;
    // the sums read the block partials of post_exp; the first sweep reads
    // post_tmp and the weights: both run after the same barrier
    for (int k = blockIdx.x; k < P.n_inst; k += gridDim.x) {
        reduce_sum(phase_args(P, k));
        __syncthreads();
    }
    for (int it = 0; it < P.max_iters; ++it) {
        for (int w = blockIdx.x; w < P.n_blocks; w += gridDim.x) {
            const PostArgs& A = phase_item(P, w, bx);
            if (it < A.iters) {
                if (A.K == 32) post_sweep<32>(A, bx, it);
                else if (A.K == 16) post_sweep<16>(A, bx, it);
                else post_sweep<0>(A, bx, it);
            }
        }
        if (!sync()) return;
    }
    if (P.max_iters == 0 && !sync()) return;   // the sums before final_part rewrites the partials
    for (int w = blockIdx.x; w < P.n_blocks; w += gridDim.x) {
        const PostArgs& A = phase_item(P, w, bx);
        final_part(A, bx);
        __syncthreads();
    }
    if (!sync()) return;
    for (int k = blockIdx.x; k < P.n_inst; k += gridDim.x) {
        final_reduce(phase_args(P, k));
        __syncthreads();
    }
    if (!sync()) return;
    for (int w = blockIdx.x; w < P.n_blocks; w += gridDim.x) {
        const PostArgs& A = phase_item(P, w, bx);
        normalise(A, bx);
    }
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
    A.lfloor = c->p.post_floor > 0.f ? -(double)c->p.post_floor : -INFINITY;
    A.poses = c->poses[c->cur];
    A.best_pose = c->best_pose;
    A.err = c->dev_error;
    return A;
}

// Resident CTAs of k_post_phase on the current device: the grid of a
// cooperative launch may not exceed it.
unsigned post_capacity() {
    static int cap[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cap[dev]) {
        int sms = 0, per = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_post_phase, PB, 0) != cudaSuccess)
            return 0;
        cap[dev] = sms * per;
    }
    return (unsigned)cap[dev];
}

long long post_budget(const mp_ctx* c) { return c->wait_budget > 0 ? c->wait_budget : MP_WAIT_BUDGET; }

}  // namespace

int mp_launch_posterior(mp_ctx* c) {
    PostPhase P = {};
    P.one = post_args(c, c->nbr_cur);
    P.n_blocks = P.one.nb;
    P.n_inst = 1;
    P.max_iters = P.one.iters;
    P.starve = c->starve_bar;
    P.bar = c->post_bar;
    P.budget = post_budget(c);
    const unsigned cap = post_capacity();
    if (!cap) return mp_fail(c, MP_ECUDA, "posterior: no resident CTAs for the cooperative launch");
    MP_CUDA(c, cudaMemsetAsync(c->post_bar, 0, sizeof(GridBar), c->stream));
    MP_CUDA(c, launch_coop((const void*)k_post_phase, std::min<unsigned>((unsigned)P.n_blocks, cap), PB, &P,
                           c->stream));
    MP_LAUNCHED(c);
    return MP_OK;
}

// Batched posterior: one cooperative launch over the particle blocks of all
// instances (its barrier zeroed first).
int mp_plan_posterior(mp_group* G, int p, std::vector<GOp>& plan) {
    std::vector<PostArgs> tab;
    std::vector<int64_t> bpb;
    int max_iters = 0;
    for (int i = 0; i < G->size(); ++i) {
        mp_ctx* c = G->ctx[i];
        tab.push_back(post_args(c, c->nbr_cur ^ p ^ 1));   // the list the merge of this step wrote
        bpb.push_back(tab.back().nb);
        max_iters = std::max(max_iters, tab.back().iters);
    }
    GridBar* bar = static_cast<GridBar*>(G->scratch(sizeof(GridBar)));
    const PostArgs* t = G->upload(tab);
    unsigned nblk = 0;
    const GBlk* map = G->block_map(bpb, &nblk);
    const unsigned cap = post_capacity();
    if (G->err) return G->err;
    if (!cap) return MP_ECUDA;
    PostPhase P = {};
    P.tab = t;
    P.blocks = map;
    P.n_blocks = (int)nblk;
    P.n_inst = G->size();
    P.max_iters = max_iters;
    P.starve = G->ctx[0]->starve_bar;
    P.bar = bar;
    P.budget = post_budget(G->ctx[0]);
    plan_memset(plan, bar, sizeof(GridBar));
    plan_coop(plan, (const void*)k_post_phase, std::min(nblk, cap), PB, P);
    return MP_OK;
}
