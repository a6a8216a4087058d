// Internal header of the MegaParticles GB300 library: context layout, device
// math shared by the kernels of this library, and the host-side launchers each
// translation unit exports. Nothing here is part of the public ABI
// (include/megaparticles.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/megaparticles.h"

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
#define MP_NSTAGES 9
#define MP_EV_RING 64       // event pairs per stage kept in flight for timing
#define MP_MAXK 32          // largest neighbour list (one warp per particle)
#define MP_COVK 16          // largest covariance neighbourhood
#define MP_GN 29            // H (21) + b (6) + log-likelihood + inlier count
#define MP_RADIX_BITS 8
#define MP_RADIX 256
#define MP_SORT_TILE 2048   // elements per radix-sort block (256 threads x 8)

// Per-step values the kernels read from device memory rather than from
// their arguments, so that a captured step can be replayed: the LSH draw (as
// T_LSH^-1 and the offset delta, Eq. 10) and the prediction's motion dT, noise
// factor and counter (Eq. 1).
struct StepDev {
    double lsh_qinv[4], lsh_R[9], lsh_tinv[3], lsh_delta[6];   // lsh_R: rotation of lsh_qinv, row-major
    float dq[4], dt[3], L[21];
    int32_t noise;
    uint32_t step;
};

struct mp_ctx {
    mp_params p;
    cudaStream_t stream;
    int device;
    char err[512];
    int64_t launches;

    // map
    int64_t n_map, n_map_valid;
    float4* map_pts;        // n_map: x, y, z, 0
    float* map_normals;     // n_map x 3
    uint8_t* map_valid;     // n_map
    float4* map_rec;        // 2 per map point, in spatial (Morton) order: (mu.xyz, n.x), (n.y, n.z, 0, 0)
    int32_t* map_perm;      // spatial order -> original index
    int32_t* nnf;           // dense voxel grid of spatial-order map indices, -1 = none within r_max
    int32_t nnf_dims[3];
    int64_t nnf_voxels;
    float nnf_origin[3], nnf_inv_res, nnf_off[3];
    double map_lo[3], map_hi[3];
    std::atomic<int>* map_refs;   // contexts using these map buffers (mp_init_map_shared); the last frees them

    // particles
    int64_t n;              // particles (0 = not initialised)
    int64_t cap;            // allocated particles
    float4* poses[2];       // 2 float4 per particle: (qx, qy, qz, qw), (tx, ty, tz, 0)
    int cur;                // current pose buffer
    double* logprior;
    double* post;
    double* post_tmp;
    double* post_init;      // unnormalised initial posterior exp(l - max l)
    double* post_invden;    // 1 / sum_j k_ij of the current lists
    double* post_w;         // k_ij / sum_j k_ij (FP64), fixed for a step's sweeps; slot-major: [l * n + i]
    int32_t* post_ids;      // the lists' ids, slot-major [l * n + i] (coalesced sweeps)
    float* loglik;
    int32_t* n_in;
    uint32_t* keys;
    uint32_t* buckets;
    int32_t* sorted_ids;
    int32_t* rank;
    int32_t* visit;         // the likelihood's visiting order (position cells, LSH order within a cell)
    int32_t* seg;           // 2 per particle
    uint32_t* sort_keys[2];
    int32_t* sort_ids[2];
    uint32_t* radix_counts; // MP_RADIX * n_sort_blocks
    uint32_t* scan_tmp;     // block sums for the scans
    size_t scan_tmp_cap;
    int32_t* nbr_ids[2];
    int nbr_cur;
    float* nbr_k;
    float* nbr_d;
    float* gn;              // MP_GN x cap, structure of arrays, sorted order
    float* psi;             // 8 floats per particle (6 used)
    float* pinv;            // 24 floats per particle: (H + lambda diag H + eps I)^-1, upper triangle
                            // (21 used); allocated when svgd_precond is set
    float* phi;             // 8 floats per particle (6 used)

    // scan
    int32_t n_scan;
    float* scan_raw;        // max_scan x 3
    float* scan_normals;    // max_scan x 3
    uint8_t* scan_valid;    // max_scan
    float4* scan_pair;      // 3 per valid point, every value twice (a broadcast pair):
                            // (mx,mx,my,my), (mz,mz,nx,nx), (ny,ny,nz,nz)
    float4* scan_tmp4;      // max_scan float4 copy of the raw scan
    int32_t* scan_nvalid;   // device scalar

    // odometry of the current step (FP32 for the kernels)
    float odom_q[4], odom_t[3];
    float chol[21];         // lower-triangular Cholesky factor of Sigma^dT (rows)
    int noise;

    // LSH draw of the current step
    double lsh_q[4], lsh_t[3], lsh_delta[6];
    uint64_t step;
    // device copy of the per-step values, filled from a ring of two pinned
    // host slots (an event per slot guards its reuse); batch_slot, when set,
    // replaces the ring (a captured step copies from a fixed slot)
    StepDev* step_dev;
    StepDev* step_host;
    cudaEvent_t step_ev[2];
    int step_ring;
    StepDev* batch_slot;

    // reductions
    double* red;            // partials
    double* scalars;        // [0] max l, [1] sum exp, [2] sum post, [3] best prob
    int64_t* best_idx;
    float4* best_pose;      // 2 float4
    int32_t* dev_error;     // bit 0: a bounded wait gave up

    // timing: a ring of event pairs per stage; totals folded in as slots recycle
    int timing;
    cudaEvent_t ev[MP_EV_RING][MP_NSTAGES][2];
    int64_t stage_runs[MP_NSTAGES];
    double stage_ms[MP_NSTAGES];
    unsigned long long* pairs;   // device counter of likelihood pairs

    // host staging
    void* host_tmp;
    size_t host_tmp_bytes;

    // test knobs of the failure path
    int precision;           // MP_PREC_* of the likelihood stage
    int lk_split;            // CTAs sharing the scan of one particle block (FP32 likelihood; 0/1 = none)
    struct GicpBufs* gicp;   // scan-to-scan odometry buffers (allocated at first use)
    uint4* scan_h2;          // 2 per valid point: the scan as 16-bit broadcast pairs (precision != FP32)
    long long wait_budget;   // cycles; 0 = MP_WAIT_BUDGET
    int starve_tx;
    int starve_bar;          // test knob: the first grid barrier of the posterior (and of a batch's sort phase) waits for one CTA more than the grid
    struct GridBar* post_bar;   // the persistent posterior's grid barrier (zeroed before each launch)
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
struct Quat {
    float x, y, z, w;
};

__device__ __forceinline__ Quat qmul(const Quat& a, const Quat& b) {
    Quat r;
    r.w = a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z;
    r.x = a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y;
    r.y = a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x;
    r.z = a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w;
    return r;
}

__device__ __forceinline__ Quat qnormalize(const Quat& a) {
    float s = rsqrtf(a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w);
    return Quat{a.x * s, a.y * s, a.z * s, a.w * s};
}

// Rotation matrix of a unit quaternion (value path; contraction allowed).
__device__ __forceinline__ void quat_rot(const Quat& q, float R[9]) {
    float x2 = q.x + q.x, y2 = q.y + q.y, z2 = q.z + q.z;
    float xx = q.x * x2, yy = q.y * y2, zz = q.z * z2;
    float xy = q.x * y2, xz = q.x * z2, yz = q.y * z2;
    float wx = q.w * x2, wy = q.w * y2, wz = q.w * z2;
    R[0] = 1.f - (yy + zz); R[1] = xy - wz; R[2] = xz + wy;
    R[3] = xy + wz; R[4] = 1.f - (xx + zz); R[5] = yz - wx;
    R[6] = xz - wy; R[7] = yz + wx; R[8] = 1.f - (xx + yy);
}

// Rotation matrix by the fixed, un-fused FP32 sequence used wherever the
// result decides an integer (the voxel of a transformed point): every product
// and sum is rounded separately (__fmul_rn/__fadd_rn/__fsub_rn forbid
// contraction).
__device__ __forceinline__ void quat_rot_exact(const Quat& q, float R[9]) {
    float x2 = __fadd_rn(q.x, q.x), y2 = __fadd_rn(q.y, q.y), z2 = __fadd_rn(q.z, q.z);
    float xx = __fmul_rn(q.x, x2), yy = __fmul_rn(q.y, y2), zz = __fmul_rn(q.z, z2);
    float xy = __fmul_rn(q.x, y2), xz = __fmul_rn(q.x, z2), yz = __fmul_rn(q.y, z2);
    float wx = __fmul_rn(q.w, x2), wy = __fmul_rn(q.w, y2), wz = __fmul_rn(q.w, z2);
    R[0] = __fsub_rn(1.f, __fadd_rn(yy, zz)); R[1] = __fsub_rn(xy, wz); R[2] = __fadd_rn(xz, wy);
    R[3] = __fadd_rn(xy, wz); R[4] = __fsub_rn(1.f, __fadd_rn(xx, zz)); R[5] = __fsub_rn(yz, wx);
    R[6] = __fsub_rn(xz, wy); R[7] = __fadd_rn(yz, wx); R[8] = __fsub_rn(1.f, __fadd_rn(xx, yy));
}

// Squared distance ((dx*dx + dy*dy) + dz*dz), dx = b.x - a.x, un-fused: the
// decision sequence of neighbourhoods and of the NNF.
__device__ __forceinline__ float dist2_exact(float ax, float ay, float az, float bx, float by, float bz) {
    float dx = __fsub_rn(bx, ax), dy = __fsub_rn(by, ay), dz = __fsub_rn(bz, az);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// floor(x) as an integer for |x| < 2^22 with one FP32 add rounded toward
// -inf: 1.5 * 2^23 + x lands in [2^23, 2^24) where the spacing is 1.
// Out-of-range or non-finite x give values far outside any grid dimension.
__device__ __forceinline__ int floor_to_int(float x) {
    return __float_as_int(__fadd_rd(x, 12582912.0f)) - 0x4B400000;
}

// 3-vector helpers
__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// exp: so(3) -> unit quaternion (FP32). sin(h)/theta and cos(h), h = theta/2,
// by their Taylor series below theta = 1e-2.
__device__ __forceinline__ Quat so3_exp_f(const float w[3], float* sinc_half_out = nullptr) {
    float th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    float s, c;
    if (th2 < 1e-4f) {
        s = 0.5f - th2 * (1.f / 48.f) + th2 * th2 * (1.f / 3840.f);
        c = 1.f - th2 * 0.125f + th2 * th2 * (1.f / 384.f);
    } else {
        float th = sqrtf(th2);
        float sh, ch;
        sincosf(0.5f * th, &sh, &ch);
        s = sh / th;
        c = ch;
    }
    if (sinc_half_out) *sinc_half_out = s;
    return Quat{s * w[0], s * w[1], s * w[2], c};
}

// SE(3) exp of xi = (omega, v): rotation and V(omega) v with
// V = I + A [w]x + B [w]x^2, A = 2 (sin(h)/theta)^2, B = (theta - sin theta)/theta^3
// (series below theta = 1).
__device__ __forceinline__ void se3_exp_f(const float xi[6], Quat& q, float t[3]) {
    float sh;
    q = so3_exp_f(xi, &sh);
    float th2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    float A = 2.f * sh * sh;
    float B;
    if (th2 < 1.f) {
        B = (1.f / 6.f) + th2 * (-1.f / 120.f + th2 * (1.f / 5040.f + th2 * (-1.f / 362880.f + th2 * (1.f / 39916800.f))));
    } else {
        float th = sqrtf(th2);
        B = (th - sinf(th)) / (th2 * th);
    }
    float wv[3], wwv[3];
    cross3(xi, xi + 3, wv);
    cross3(xi, wv, wwv);
    t[0] = xi[3] + A * wv[0] + B * wwv[0];
    t[1] = xi[4] + A * wv[1] + B * wwv[1];
    t[2] = xi[5] + A * wv[2] + B * wwv[2];
}

// SE(3) log of (q, t): omega = 2 atan2(|v|, w) v/|v| (w >= 0), and
// V^-1(omega) t = t - 1/2 w x t + C w x (w x t),
// C = (1 - (theta/2) cot(theta/2)) / theta^2 (series below theta = 1).
__device__ __forceinline__ void se3_log_f(Quat q, const float t[3], float xi[6]) {
    if (q.w < 0.f) { q.x = -q.x; q.y = -q.y; q.z = -q.z; q.w = -q.w; }
    float s2 = q.x * q.x + q.y * q.y + q.z * q.z;
    float f;
    if (s2 < 1e-8f) {
        f = 2.f / q.w * (1.f - s2 / (3.f * q.w * q.w));
    } else {
        float s = sqrtf(s2);
        f = 2.f * atan2f(s, q.w) / s;
    }
    xi[0] = f * q.x; xi[1] = f * q.y; xi[2] = f * q.z;
    float th2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
    float C;
    if (th2 < 1.f) {
        C = (1.f / 12.f) + th2 * (1.f / 720.f + th2 * (1.f / 30240.f + th2 * (1.f / 1209600.f)));
    } else {
        float th = sqrtf(th2);
        float sh, ch;
        sincosf(0.5f * th, &sh, &ch);
        C = (1.f - 0.5f * th * ch / sh) / th2;
    }
    float wt[3], wwt[3];
    cross3(xi, t, wt);
    cross3(xi, wt, wwt);
    xi[3] = t[0] - 0.5f * wt[0] + C * wwt[0];
    xi[4] = t[1] - 0.5f * wt[1] + C * wwt[1];
    xi[5] = t[2] - 0.5f * wt[2] + C * wwt[2];
}

__device__ __forceinline__ void rot_apply(const float R[9], const float v[3], float o[3]) {
    o[0] = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
    o[1] = R[3] * v[0] + R[4] * v[1] + R[5] * v[2];
    o[2] = R[6] * v[0] + R[7] * v[1] + R[8] * v[2];
}
__device__ __forceinline__ void rot_apply_T(const float R[9], const float v[3], float o[3]) {
    o[0] = R[0] * v[0] + R[3] * v[1] + R[6] * v[2];
    o[1] = R[1] * v[0] + R[4] * v[1] + R[7] * v[2];
    o[2] = R[2] * v[0] + R[5] * v[1] + R[8] * v[2];
}

// (q, t) <- (q, t) exp(xi), renormalised.
__device__ __forceinline__ void pose_retract(Quat& q, float t[3], const float xi[6]) {
    Quat dq;
    float dt[3], R[9], Rdt[3];
    se3_exp_f(xi, dq, dt);
    quat_rot(q, R);
    rot_apply(R, dt, Rdt);
    t[0] += Rdt[0]; t[1] += Rdt[1]; t[2] += Rdt[2];
    q = qnormalize(qmul(q, dq));
}

__device__ __forceinline__ void load_pose(const float4* poses, int64_t i, Quat& q, float t[3]) {
    float4 a = poses[2 * i], b = poses[2 * i + 1];
    q = Quat{a.x, a.y, a.z, a.w};
    t[0] = b.x; t[1] = b.y; t[2] = b.z;
}
// 32 bytes (two float4, 32-byte aligned, read-only for the whole kernel) in
// one 256-bit load.
__device__ __forceinline__ void ld_nc_2x4(const float4* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}
__device__ __forceinline__ void store_pose(float4* poses, int64_t i, const Quat& q, const float t[3]) {
    poses[2 * i] = make_float4(q.x, q.y, q.z, q.w);
    poses[2 * i + 1] = make_float4(t[0], t[1], t[2], 0.f);
}

// Philox-4x32-10 (Salmon et al., SC 2011): ten rounds, two 32x32 multiplies
// per round, Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}
#define MP_STREAM_PREDICT 1u
#define MP_STREAM_LSH 2u
#define MP_STREAM_INIT 3u

// (x + 1/2) / 2^32 in FP32
__device__ __forceinline__ float u32_to_open01(uint32_t x) {
    return fmaf((float)x, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy (TMA) helpers. Waits are bounded: on expiry the caller
// records an error and stops.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Orders this CTA's earlier generic-proxy accesses to shared memory (made
// visible to the issuing thread by a barrier) before its later async-proxy
// (bulk copy) writes: the write-after-read order of a reused staging buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Spin on the barrier phase for at most `budget` SM clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long budget) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}
#define MP_WAIT_BUDGET (4000000000LL)   // ~2 s at 2 GHz
#define MP_ERR_WAIT 1

// Grid-wide barrier of a cooperative (persistent) launch, whose CTAs are all
// resident at once. Thread 0 of each CTA reads the generation, arrives on the
// counter and, unless it is the last to arrive, spins until the generation
// moves on; the last arrival resets the counter and advances the generation.
// The spin is bounded by `budget` SM cycles and also ends when another CTA has
// given up (abort); grid_sync then returns false and the caller records the
// error and returns. Zero the barrier before every launch.
struct GridBar {
    unsigned int count, gen;
    int abort, pad;
};
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ bool grid_sync(GridBar* gb, unsigned expected, long long budget) {
    __shared__ int ok_s;
    __syncthreads();   // the CTA's share of the sub-step is done
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire_u32(&gb->gen);
        __threadfence();   // this CTA's writes before its arrival
        if (atomicAdd(&gb->count, 1u) + 1u == expected) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire_u32(&gb->gen) == g) {
                if (ld_relaxed_s32(&gb->abort) != 0 || clock64() - t0 > budget) {
                    ok = 0;
                    atomicExch(&gb->abort, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();   // the other CTAs' writes after the barrier
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// ---------------------------------------------------------------------------
// host-side helpers
// ---------------------------------------------------------------------------
int mp_fail(mp_ctx* c, int code, const char* fmt, ...);
// records the message of a failure without a context (mp_last_error(NULL))
int mp_fail_noctx(int code, const char* fmt, ...);
int mp_cuda_check(mp_ctx* c, cudaError_t e, const char* what);
#define MP_CUDA(ctx, call)                                              \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return mp_cuda_check((ctx), _e, #call);  \
    } while (0)
// Checked builds (-DMP_CHECKED; a debugging aid, see build.py): kernels test
// the indices they take from data (neighbour ids, map indices, sort positions,
// the scan chunk bounds) before using them, print each violation and skip the
// access; on the host every launch outside a stream capture is synchronised,
// so that a fault is reported at the launch that caused it. In normal builds
// both macros compile to nothing.
#if defined(MP_CHECKED) && defined(MP_CHECKED_LITE)
// The light form (-DMP_CHECKED_LITE, build(checked="lite")): a violation
// records its source line in a per-file device word with one atomic and
// skips the access (no printf: the kernels' code stays close to the normal
// build's); after every synchronised launch the host reads the file's word.
static __device__ unsigned int mp_dcheck_line;
#define MP_DCHECK(cond, what, v) ((cond) ? true : (atomicCAS(&mp_dcheck_line, 0u, (unsigned)__LINE__), false))
int mp_checked_sync(mp_ctx* c, const char* file, int line);
static inline int mp_dcheck_poll(mp_ctx* c, const char* file, int line) {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, mp_dcheck_line, sizeof(v)) != cudaSuccess) return MP_OK;
    if (v) {
        fprintf(stderr, "MP_CHECKED %s:%u: index check fired (kernel launched at line %d)\n", file, v, line);
        return mp_fail(c, MP_ECUDA, "index check at %s:%u", file, v);
    }
    return MP_OK;
}
#define MP_CHECKED_SYNC(ctx)                                          \
    do {                                                              \
        int _r = mp_checked_sync((ctx), __FILE__, __LINE__);          \
        if (!_r) _r = mp_dcheck_poll((ctx), __FILE__, __LINE__);      \
        if (_r) return _r;                                            \
    } while (0)
#elif defined(MP_CHECKED)
#define MP_DCHECK(cond, what, v)                                                                        \
    ((cond) ? true                                                                                      \
            : (printf("MP_CHECKED %s:%d: %s (%lld) block %d thread %d\n", __FILE__, __LINE__, what,      \
                      (long long)(v), (int)blockIdx.x, (int)threadIdx.x),                               \
               false))
int mp_checked_sync(mp_ctx* c, const char* file, int line);
#define MP_CHECKED_SYNC(ctx)                                          \
    do {                                                              \
        int _r = mp_checked_sync((ctx), __FILE__, __LINE__);          \
        if (_r) return _r;                                            \
    } while (0)
#else
#define MP_DCHECK(cond, what, v) true
#define MP_CHECKED_SYNC(ctx) \
    do {                     \
    } while (0)
#endif
#define MP_LAUNCHED(ctx)                                                           \
    do {                                                                           \
        (ctx)->launches++;                                                         \
        cudaError_t _e = cudaGetLastError();                                       \
        if (_e != cudaSuccess) return mp_cuda_check((ctx), _e, "kernel launch");   \
        MP_CHECKED_SYNC(ctx);                                                      \
    } while (0)

static inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// launchers (each returns MP_OK or an error code recorded in ctx)
// k_map.cu
void draw_lsh(mp_ctx* c);
void odom_to_pose_host(const double T[16], double q[4], double t[3]);   // identity for NULL
void mp_gicp_free(mp_ctx* c);
void fill_step_host(mp_ctx* c, StepDev* h);
int upload_step(mp_ctx* c);
int mp_launch_map_prepare(mp_ctx* c, const float* xyz_dev);
int mp_launch_scan_prepare(mp_ctx* c);
int mp_launch_point_gaussians(mp_ctx* c, const float* raw_dev, int n, float4* tmp4, float* normals, uint8_t* valid);
int mp_launch_nnf_query(mp_ctx* c, const int32_t* vox_dev, int64_t m, int32_t* out_dev);
// k_neighbors.cu
int mp_launch_lsh_keys(mp_ctx* c);
int mp_launch_sort(mp_ctx* c);
int mp_launch_merge(mp_ctx* c);
int mp_launch_exclusive_scan(mp_ctx* c, const uint32_t* in, uint32_t* out, int64_t n);
// k_likelihood.cu
int mp_launch_likelihood(mp_ctx* c);
// k_update.cu
int mp_launch_predict(mp_ctx* c);
int mp_launch_solve(mp_ctx* c);
int mp_launch_svgd(mp_ctx* c);
int mp_launch_init_uniform(mp_ctx* c, const float lo[6], const float hi[6]);
int mp_launch_pack_poses(mp_ctx* c, const float* src7_dev, float4* dst);
int mp_launch_unpack_poses(mp_ctx* c, const float4* src, float* dst7_dev);
int mp_launch_gather_gn(mp_ctx* c, float* dst_dev);
// k_posterior.cu
int mp_launch_posterior(mp_ctx* c);
// k_pn_tc.cu: the proposal network's fused per-point layers on the tensor cores
size_t mp_pn_tc_image_bytes();
int mp_pn_tc_pack(const float* W2, const float* W3, uint8_t* image, cudaStream_t s);
int mp_pn_tc_forward(const float* xs, int B, int P, const float* W1, const float* b1, const float* b2,
                     const float* b3, const uint8_t* image, float* g, int* gi, float* h1_out, float* h2_out,
                     int32_t* err, long long budget, cudaStream_t s);

// ---------------------------------------------------------------------------
// grouped launches (batched instances, mp_batch_*): one kernel over the blocks
// of many instances. Block b of a grouped launch runs block (map[b].bx,
// map[b].by) of instance map[b].inst with that instance's argument record
// tab[map[b].inst], through the same body (Op::run) as the instance's own
// launch, so a grouped phase computes what the per-instance launches compute.
// ---------------------------------------------------------------------------
struct GBlk {
    int32_t inst, bx, by, pad;
};

template <typename Op>
__global__ void __launch_bounds__(Op::THREADS, Op::MINB) k_group(const typename Op::Args* __restrict__ tab,
                                                               const GBlk* __restrict__ map) {
    const GBlk g = map[blockIdx.x];
    Op::run(tab[g.inst], (unsigned)g.bx, (unsigned)g.by);
}

// One operation of a batch step's plan: a grouped kernel (func = k_group<Op>,
// arguments tab and map, grid blocks of block threads), a cooperative
// persistent kernel (func with one by-value argument of arg_bytes in arg), a
// device memset or a device-to-device copy. The plan is captured into a CUDA
// graph.
struct GOp {
    enum Kind { KERNEL, COOP, MEMSET, COPY } kind;
    const void* func;
    unsigned grid, block;
    const void* tab;
    const GBlk* map;
    void* dst;
    const void* src;
    size_t bytes;
    size_t arg_bytes;
    alignas(16) unsigned char arg[512];
};

// The instances of a batch as the planners see them: contexts, the device
// copies of the step inputs (all scans in one buffer, one StepDev each), and
// the device tables the plans point to (freed with the group).
struct mp_group {
    std::vector<mp_ctx*> ctx;
    std::vector<int32_t> n_scan;
    std::vector<int64_t> scan_off;   // floats into scan_dev
    float* scan_dev = nullptr;
    StepDev* sd_dev = nullptr;
    std::vector<void*> arena;
    int err = 0;                     // first allocation / copy error (MP_ENOMEM / MP_ECUDA)

    int size() const { return (int)ctx.size(); }
    // device copy of a host array (nullptr and err set on failure)
    const void* upload(const void* host, size_t bytes);
    // zeroed device memory the plan's kernels write (nullptr and err set on failure)
    void* scratch(size_t bytes);
    template <typename T>
    const T* upload(const std::vector<T>& v) {
        return static_cast<const T*>(upload(v.data(), sizeof(T) * v.size()));
    }
    // block map over the instances in `which` (all when empty): instance i
    // gets blocks[i] x ysplit[i] blocks (ysplit empty = 1); *nblk = total
    const GBlk* block_map(const std::vector<int64_t>& blocks, unsigned* nblk, const std::vector<int>& which = {},
                          const std::vector<int>& ysplit = {});
    void release();
};

// Appends a grouped kernel to a plan (nothing when no instance has blocks).
template <typename Op>
inline void plan_kernel(std::vector<GOp>& plan, const typename Op::Args* tab, const GBlk* map, unsigned nblk) {
    if (nblk == 0 || !tab || !map) return;
    GOp o{};
    o.kind = GOp::KERNEL;
    o.func = reinterpret_cast<const void*>(&k_group<Op>);
    o.grid = nblk;
    o.block = Op::THREADS;
    o.tab = tab;
    o.map = map;
    plan.push_back(o);
}
// Appends a cooperative launch of func(arg) (grid <= the resident CTAs).
template <typename T>
inline void plan_coop(std::vector<GOp>& plan, const void* func, unsigned grid, unsigned block, const T& arg) {
    static_assert(sizeof(T) <= sizeof(GOp::arg), "argument too large");
    if (grid == 0) return;
    GOp o{};
    o.kind = GOp::COOP;
    o.func = func;
    o.grid = grid;
    o.block = block;
    o.arg_bytes = sizeof(T);
    memcpy(o.arg, &arg, sizeof(T));
    plan.push_back(o);
}
// A cooperative launch on a stream (also inside a stream capture).
inline cudaError_t launch_coop(const void* func, unsigned grid, unsigned block, void* arg, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    void* args[1] = {arg};
    return cudaLaunchKernelExC(&cfg, func, args);
}
inline void plan_memset(std::vector<GOp>& plan, void* dst, size_t bytes) {
    GOp o{};
    o.kind = GOp::MEMSET;
    o.dst = dst;
    o.bytes = bytes;
    plan.push_back(o);
}
inline void plan_copy(std::vector<GOp>& plan, void* dst, const void* src, size_t bytes) {
    GOp o{};
    o.kind = GOp::COPY;
    o.dst = dst;
    o.src = src;
    o.bytes = bytes;
    plan.push_back(o);
}

// Planners: the grouped launches of one stage for neighbour-list parity p.
// They run while every context still has the list index nbr_cur0 it had when
// the batch was created: graph p's merge reads list nbr_cur0 ^ p and writes
// nbr_cur0 ^ p ^ 1, which SVGD and the posterior then read. Each returns
// MP_OK or the group's error.
int mp_plan_predict(mp_group* G, int p, std::vector<GOp>& plan);
int mp_plan_scan(mp_group* G, int p, std::vector<GOp>& plan);
int mp_plan_lsh_sort(mp_group* G, int p, std::vector<GOp>& plan);
int mp_plan_merge(mp_group* G, int p, std::vector<GOp>& plan);
int mp_plan_likelihood(mp_group* G, int p, std::vector<GOp>& plan);
int mp_plan_solve_svgd(mp_group* G, int p, std::vector<GOp>& plan);
int mp_plan_posterior(mp_group* G, int p, std::vector<GOp>& plan);
