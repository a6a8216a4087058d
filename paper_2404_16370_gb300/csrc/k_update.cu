// Particle-state kernels:
//  * k_predict  Sec. III-B, Eq. 1: T_i <- T_i dT exp(L n_i), n_i ~ N(0, I) by
//               Box-Muller on Philox(seed; i, {0,1}, step, PREDICT).
//  * k_solve    Sec. III-C: psi_i = -(H + lambda diag H + eps I)^-1 b, FP64
//               LDL^T (psi = 0 below 6 inliers or on a non-positive pivot).
//  * k_svgd     Sec. III-C, Eq. 5-6: phi_i = sum_j (k_ij psi_j - 2 k_ij W d_ij) /
//               sum_j k_ij over the list of i; T_i <- T_i exp(phi_i). A group
//               of lanes per particle (one per list slot), shuffle reductions.
//               With svgd_precond the repulsive sum is multiplied by the
//               particle's damped Gauss-Newton inverse, which k_solve stores.
//  * k_init     uniform particle draws (Sec. IV-A).
//  * pose (un)packing between the ABI layout (7 floats) and 2 x float4.
#include "mp_internal.cuh"

namespace {

struct PredArgs {
    float4* poses;
    int64_t n;
    uint2 key;
    const StepDev* sd;   // the motion dT, the noise factor and the step counter (replayable)
};

struct PredOp {
    using Args = PredArgs;
    static constexpr int THREADS = 256, MINB = 1;
    static __device__ __forceinline__ void run(const PredArgs& A, unsigned bx, unsigned);
};

__device__ __forceinline__ void PredOp::run(const PredArgs& A, unsigned bx, unsigned) {
    const StepDev* __restrict__ sd = A.sd;
    int64_t i = (int64_t)bx * THREADS + threadIdx.x;
    if (i >= A.n) return;
    Quat q;
    float t[3];
    load_pose(A.poses, i, q, t);
    // T dT
    float R[9], r[3];
    quat_rot(q, R);
    const float dt[3] = {sd->dt[0], sd->dt[1], sd->dt[2]};
    rot_apply(R, dt, r);
    t[0] += r[0]; t[1] += r[1]; t[2] += r[2];
    q = qmul(q, Quat{sd->dq[0], sd->dq[1], sd->dq[2], sd->dq[3]});
    if (sd->noise) {
        const uint32_t step = sd->step;
        uint4 o0 = philox4x32_10(make_uint4((uint32_t)i, 0u, step, MP_STREAM_PREDICT), A.key);
        uint4 o1 = philox4x32_10(make_uint4((uint32_t)i, 1u, step, MP_STREAM_PREDICT), A.key);
        uint32_t u[6] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y};
        float z[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float rad = sqrtf(-2.f * logf(u32_to_open01(u[2 * k])));
            float s, cs;
            sincospif(2.f * u32_to_open01(u[2 * k + 1]), &s, &cs);
            z[2 * k] = rad * cs;
            z[2 * k + 1] = rad * s;
        }
        float xi[6];
        int o = 0;
#pragma unroll
        for (int rr = 0; rr < 6; ++rr) {
            float s = 0.f;
#pragma unroll
            for (int cc = 0; cc <= rr; ++cc) s += sd->L[o++] * z[cc];
            xi[rr] = s;
        }
        pose_retract(q, t, xi);
    } else {
        q = qnormalize(q);
    }
    store_pose(A.poses, i, q, t);
}

__global__ void __launch_bounds__(256) k_predict(const PredArgs A) { PredOp::run(A, blockIdx.x, 0); }

struct SolveArgs {
    const float* gn;
    int64_t stride;
    const int32_t* order;
    int64_t n;
    double lambda, eps;
    float* psi;
    float* loglik;
    int32_t* n_in;
    float* pinv;   // nullptr: no inverse stored
};

struct SolveOp {
    using Args = SolveArgs;
    static constexpr int THREADS = 128, MINB = 1;
    static __device__ __forceinline__ void run(const SolveArgs& A, unsigned bx, unsigned);
};

__device__ __forceinline__ void SolveOp::run(const SolveArgs& args, unsigned bx, unsigned) {
    const float* __restrict__ gn = args.gn;
    const int64_t stride = args.stride, n = args.n;
    const int32_t* __restrict__ order = args.order;
    const double lambda = args.lambda, eps = args.eps;
    float* __restrict__ psi = args.psi;
    float* __restrict__ loglik = args.loglik;
    int32_t* __restrict__ n_in = args.n_in;
    float* __restrict__ pinv = args.pinv;
    int64_t p = (int64_t)bx * THREADS + threadIdx.x;
    if (p >= n) return;
    int64_t i = order[p];
    if (!MP_DCHECK(i >= 0 && i < n, "particle order entry", i)) return;
    double A[6][6];
    int o = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) {
            double v = gn[(int64_t)o++ * stride + p];
            A[r][c] = v;
            A[c][r] = v;
        }
    double b[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) b[r] = gn[(int64_t)(21 + r) * stride + p];
    float ll = gn[27 * stride + p];
    int cnt = (int)gn[28 * stride + p];
#pragma unroll
    for (int r = 0; r < 6; ++r) A[r][r] = A[r][r] + fma(lambda, A[r][r], eps);
    // LDL^T in place: strictly lower part holds L, diagonal holds D
    bool good = cnt >= 6;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        double d = A[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) d = fma(-A[j][k] * A[j][k], A[k][k], d);
        good = good && (d > 0.0);
        A[j][j] = d;
        double inv = good ? 1.0 / d : 0.0;
#pragma unroll
        for (int r = j + 1; r < 6; ++r) {
            double s = A[r][j];
#pragma unroll
            for (int k = 0; k < j; ++k) s = fma(-A[r][k] * A[j][k], A[k][k], s);
            A[r][j] = s * inv;
        }
    }
    double x[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        double s = -b[r];
#pragma unroll
        for (int k = 0; k < r; ++k) s = fma(-A[r][k], x[k], s);
        x[r] = s;
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) x[r] = good ? x[r] / A[r][r] : 0.0;
#pragma unroll
    for (int r = 5; r >= 0; --r) {
        double s = x[r];
#pragma unroll
        for (int k = r + 1; k < 6; ++k) s = fma(-A[k][r], x[k], s);
        x[r] = s;
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) psi[i * 8 + r] = good ? (float)x[r] : 0.f;
    if (pinv) {
        // the damped matrix's inverse from the same factors, column by column
        // (upper triangle stored); zero when no step was taken
        int oo = 0;
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) {
            double z[6];
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                double v = r == cc ? 1.0 : 0.0;
#pragma unroll
                for (int k = 0; k < r; ++k) v = fma(-A[r][k], z[k], v);
                z[r] = v;
            }
#pragma unroll
            for (int r = 0; r < 6; ++r) z[r] = good ? z[r] / A[r][r] : 0.0;
#pragma unroll
            for (int r = 5; r >= 0; --r) {
                double v = z[r];
#pragma unroll
                for (int k = r + 1; k < 6; ++k) v = fma(-A[k][r], z[k], v);
                z[r] = v;
            }
#pragma unroll
            for (int r = 0; r <= cc; ++r) pinv[i * 24 + oo++] = good ? (float)z[r] : 0.f;
        }
    }
    loglik[i] = ll;
    n_in[i] = cnt;
}

__global__ void __launch_bounds__(128) k_solve(const SolveArgs A) { SolveOp::run(A, blockIdx.x, 0); }

struct SvgdArgs {
    float4* poses;
    int64_t n;
    int K;
    const int32_t* ids;
    const float* kk;
    const float* dd;
    const float* psi;
    float wr, wt;
    const float* pinv;
    float* phi;
};

// G lanes per particle (G = power of two >= K, <= 32)
template <int G, bool PRE>
struct SvgdOp {
    using Args = SvgdArgs;
    static constexpr int THREADS = 256, MINB = 1;
    static __device__ __forceinline__ void run(const SvgdArgs& A, unsigned bx, unsigned);
};

template <int G, bool PRE>
__device__ __forceinline__ void SvgdOp<G, PRE>::run(const SvgdArgs& A, unsigned bx, unsigned) {
    float4* __restrict__ poses = A.poses;
    const int64_t n = A.n;
    const int K = A.K;
    const int32_t* __restrict__ ids = A.ids;
    const float* __restrict__ kk = A.kk;
    const float* __restrict__ dd = A.dd;
    const float* __restrict__ psi = A.psi;
    const float wr = A.wr, wt = A.wt;
    const float* __restrict__ pinv = A.pinv;
    float* __restrict__ phi_out = A.phi;
    // PRE: the attraction (6), the repulsion (6) and the kernel sum are
    // reduced apart, and the repulsion is multiplied by pinv_i
    constexpr int NA = PRE ? 13 : 7;
    int64_t gt = (int64_t)bx * THREADS + threadIdx.x;
    int64_t i = gt / G;
    int l = (int)(gt % G);
    bool active = i < n;
    float acc[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) acc[a] = 0.f;
    if (active && l < K) {
        int64_t o = i * K + l;
        int j = ids[o];
        if (j >= 0 && MP_DCHECK(j < n, "neighbour id", j)) {
            float k = kk[o];
            const float* dj = dd + o * 6;
            float4 p0, p1;
            ld_nc_2x4(reinterpret_cast<const float4*>(psi + (int64_t)j * 8), p0, p1);   // psi_j: one 32-byte load
            const float ps[6] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y};
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                float w = a < 3 ? wr : wt;
                if (PRE) {
                    acc[a] = k * ps[a];
                    acc[6 + a] = -2.f * k * w * dj[a];
                } else {
                    acc[a] = k * ps[a] - 2.f * k * w * dj[a];
                }
            }
            acc[NA - 1] = k;
        }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
        for (int a = 0; a < NA; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], off, G);
    if (!active || l != 0) return;
    float xi[6];
    float inv = acc[NA - 1] > 0.f ? 1.f / acc[NA - 1] : 0.f;
    if (PRE) {
        float P[21];
#pragma unroll
        for (int e = 0; e < 21; ++e) P[e] = pinv[i * 24 + e];
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            float r = 0.f;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                // upper triangle stored column by column: (r, c), r <= c at c (c + 1) / 2 + r
                const int e = a <= c ? c * (c + 1) / 2 + a : a * (a + 1) / 2 + c;
                r += P[e] * acc[6 + c];
            }
            xi[a] = (acc[a] + r) * inv;
        }
    } else {
#pragma unroll
        for (int a = 0; a < 6; ++a) xi[a] = acc[a] * inv;
    }
    Quat q;
    float t[3];
    load_pose(poses, i, q, t);
    pose_retract(q, t, xi);
    store_pose(poses, i, q, t);
#pragma unroll
    for (int a = 0; a < 6; ++a) phi_out[i * 8 + a] = xi[a];
}

template <int G, bool PRE>
__global__ void __launch_bounds__(256) k_svgd(const SvgdArgs A) { SvgdOp<G, PRE>::run(A, blockIdx.x, 0); }

struct InitArgs {
    float4* poses;
    int64_t n;
    float lo[6], hi[6];
    int full;
    uint2 key;
};

__global__ void k_init_uniform(const InitArgs A) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    uint4 o0 = philox4x32_10(make_uint4((uint32_t)i, 0u, 0u, MP_STREAM_INIT), A.key);
    uint4 o1 = philox4x32_10(make_uint4((uint32_t)i, 1u, 0u, MP_STREAM_INIT), A.key);
    float u[6] = {u32_to_open01(o0.x), u32_to_open01(o0.y), u32_to_open01(o0.z), u32_to_open01(o0.w),
                  u32_to_open01(o1.x), u32_to_open01(o1.y)};
    float v[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) v[a] = fmaf(u[a], A.hi[a] - A.lo[a], A.lo[a]);
    Quat q;
    if (A.full) {
        float a = sqrtf(1.f - u[3]), b = sqrtf(u[3]);
        float s1, c1, s2, c2;
        sincospif(2.f * u[4], &s1, &c1);
        sincospif(2.f * u[5], &s2, &c2);
        q = Quat{a * s1, a * c1, b * s2, b * c2};
    } else {
        float sr, cr, sp, cp, sy, cy;
        sincosf(0.5f * v[3], &sr, &cr);
        sincosf(0.5f * v[4], &sp, &cp);
        sincosf(0.5f * v[5], &sy, &cy);
        q = qmul(Quat{0.f, 0.f, sy, cy}, qmul(Quat{0.f, sp, 0.f, cp}, Quat{sr, 0.f, 0.f, cr}));
    }
    q = qnormalize(q);
    float t[3] = {v[0], v[1], v[2]};
    store_pose(A.poses, i, q, t);
}

__global__ void k_pack(const float* __restrict__ src, int64_t n, float4* __restrict__ dst) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    // stored exactly as given: the voxel decisions use these FP32 values
    const float* s = src + 7 * i;
    dst[2 * i] = make_float4(s[0], s[1], s[2], s[3]);
    dst[2 * i + 1] = make_float4(s[4], s[5], s[6], 0.f);
}

__global__ void k_unpack(const float4* __restrict__ src, int64_t n, float* __restrict__ dst) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 a = src[2 * i], b = src[2 * i + 1];
    float* d = dst + 7 * i;
    d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w; d[4] = b.x; d[5] = b.y; d[6] = b.z;
}

__global__ void k_gather_gn(const float* __restrict__ gn, int64_t stride, const int32_t* __restrict__ order, int64_t n,
                            float* __restrict__ dst) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t i = order[p];
    for (int f = 0; f < MP_GN; ++f) dst[i * MP_GN + f] = gn[(int64_t)f * stride + p];
}

}  // namespace

namespace {

PredArgs pred_args(mp_ctx* c, const StepDev* sd) {
    PredArgs A;
    A.poses = c->poses[c->cur];
    A.n = c->n;
    A.key = make_uint2((uint32_t)c->p.seed, (uint32_t)(c->p.seed >> 32));
    A.sd = sd;
    return A;
}

SolveArgs solve_args(mp_ctx* c) {
    SolveArgs A;
    A.gn = c->gn;
    A.stride = c->cap;
    A.order = c->visit;   // the likelihood's sums sit at its visiting slots
    A.n = c->n;
    A.lambda = (double)c->p.lambda;
    A.eps = (double)c->p.eps;
    A.psi = c->psi;
    A.loglik = c->loglik;
    A.n_in = c->n_in;
    A.pinv = c->p.svgd_precond ? c->pinv : nullptr;
    return A;
}

SvgdArgs svgd_args(mp_ctx* c, int nbr_cur) {
    SvgdArgs A;
    A.poses = c->poses[c->cur];
    A.n = c->n;
    A.K = c->p.K;
    A.ids = c->nbr_ids[nbr_cur];
    A.kk = c->nbr_k;
    A.dd = c->nbr_d;
    A.psi = c->psi;
    A.wr = c->p.sigma_r;
    A.wt = c->p.sigma_t;
    A.pinv = c->p.svgd_precond ? c->pinv : nullptr;
    A.phi = c->phi;
    return A;
}

// lanes per particle: the power of two >= K
int svgd_lanes(int K) {
    int g = 1;
    while (g < K && g < 32) g *= 2;
    return g;
}

template <int G>
int launch_svgd_g(mp_ctx* c) {
    const unsigned grid = grid_for(c->n * G, 256);
    if (c->p.svgd_precond) k_svgd<G, true><<<grid, 256, 0, c->stream>>>(svgd_args(c, c->nbr_cur));
    else k_svgd<G, false><<<grid, 256, 0, c->stream>>>(svgd_args(c, c->nbr_cur));
    MP_LAUNCHED(c);
    return MP_OK;
}

template <int G>
void plan_svgd_g(mp_group* Gr, int p, std::vector<GOp>& plan, bool pre) {
    std::vector<SvgdArgs> tab;
    std::vector<int64_t> blocks;
    std::vector<int> which;
    for (int i = 0; i < Gr->size(); ++i) {
        mp_ctx* c = Gr->ctx[i];
        tab.push_back(svgd_args(c, c->nbr_cur ^ p ^ 1));   // the list the merge of this step wrote
        blocks.push_back((c->n * G + 255) / 256);
        if (svgd_lanes(c->p.K) == G && (c->p.svgd_precond != 0) == pre) which.push_back(i);
    }
    if (which.empty()) return;
    unsigned nblk = 0;
    const GBlk* map = Gr->block_map(blocks, &nblk, which);
    const SvgdArgs* t = Gr->upload(tab);
    if (pre) plan_kernel<SvgdOp<G, true>>(plan, t, map, nblk);
    else plan_kernel<SvgdOp<G, false>>(plan, t, map, nblk);
}

}  // namespace

int mp_launch_predict(mp_ctx* c) {
    k_predict<<<grid_for(c->n, 256), 256, 0, c->stream>>>(pred_args(c, c->step_dev));
    MP_LAUNCHED(c);
    return MP_OK;
}

int mp_launch_solve(mp_ctx* c) {
    k_solve<<<grid_for(c->n, 128), 128, 0, c->stream>>>(solve_args(c));
    MP_LAUNCHED(c);
    return MP_OK;
}

int mp_launch_svgd(mp_ctx* c) {
    switch (svgd_lanes(c->p.K)) {
        case 1: return launch_svgd_g<1>(c);
        case 2: return launch_svgd_g<2>(c);
        case 4: return launch_svgd_g<4>(c);
        case 8: return launch_svgd_g<8>(c);
        case 16: return launch_svgd_g<16>(c);
        default: return launch_svgd_g<32>(c);
    }
}

int mp_plan_predict(mp_group* G, int, std::vector<GOp>& plan) {
    std::vector<PredArgs> tab;
    std::vector<int64_t> blocks;
    for (int i = 0; i < G->size(); ++i) {
        tab.push_back(pred_args(G->ctx[i], G->sd_dev + i));
        blocks.push_back((G->ctx[i]->n + 255) / 256);
    }
    unsigned nblk = 0;
    const GBlk* map = G->block_map(blocks, &nblk);
    plan_kernel<PredOp>(plan, G->upload(tab), map, nblk);
    return G->err;
}

int mp_plan_solve_svgd(mp_group* G, int p, std::vector<GOp>& plan) {
    std::vector<SolveArgs> tab;
    std::vector<int64_t> blocks;
    for (int i = 0; i < G->size(); ++i) {
        tab.push_back(solve_args(G->ctx[i]));
        blocks.push_back((G->ctx[i]->n + 127) / 128);
    }
    unsigned nblk = 0;
    const GBlk* map = G->block_map(blocks, &nblk);
    plan_kernel<SolveOp>(plan, G->upload(tab), map, nblk);
    for (int pre = 0; pre < 2; ++pre) {
        plan_svgd_g<1>(G, p, plan, pre);
        plan_svgd_g<2>(G, p, plan, pre);
        plan_svgd_g<4>(G, p, plan, pre);
        plan_svgd_g<8>(G, p, plan, pre);
        plan_svgd_g<16>(G, p, plan, pre);
        plan_svgd_g<32>(G, p, plan, pre);
    }
    return G->err;
}

int mp_launch_init_uniform(mp_ctx* c, const float lo[6], const float hi[6]) {
    InitArgs A;
    A.poses = c->poses[c->cur];
    A.n = c->n;
    const float two_pi = 6.2831853f;
    A.full = 1;
    for (int a = 0; a < 6; ++a) {
        A.lo[a] = lo[a];
        A.hi[a] = hi[a];
        if (a >= 3 && (double)hi[a] - (double)lo[a] < 6.283185307179586 - 1e-6) A.full = 0;
    }
    (void)two_pi;
    A.key = make_uint2((uint32_t)c->p.seed, (uint32_t)(c->p.seed >> 32));
    k_init_uniform<<<grid_for(c->n, 256), 256, 0, c->stream>>>(A);
    MP_LAUNCHED(c);
    return MP_OK;
}

int mp_launch_pack_poses(mp_ctx* c, const float* src7_dev, float4* dst) {
    k_pack<<<grid_for(c->n, 256), 256, 0, c->stream>>>(src7_dev, c->n, dst);
    MP_LAUNCHED(c);
    return MP_OK;
}

int mp_launch_unpack_poses(mp_ctx* c, const float4* src, float* dst7_dev) {
    k_unpack<<<grid_for(c->n, 256), 256, 0, c->stream>>>(src, c->n, dst7_dev);
    MP_LAUNCHED(c);
    return MP_OK;
}

int mp_launch_gather_gn(mp_ctx* c, float* dst_dev) {
    k_gather_gn<<<grid_for(c->n, 256), 256, 0, c->stream>>>(c->gn, c->cap, c->visit, c->n, dst_dev);
    MP_LAUNCHED(c);
    return MP_OK;
}
