// Likelihood evaluation and Gauss-Newton sums (Sec. III-C, Eq. 2-4).
//
// For particle T = (R, t) and scan point k (mu_k, normal n_k):
//   q~ = R mu_k, q = q~ + t; voxel v = floor(fma(q, 1/res, -o/res)) (FP32, the
//   fixed decision sequence); m = nnf[v] (-1 outside the grid or empty);
//   e = mu^M_m - q; Omega = (Sigma^M_m + R Sigma^S_k R^T)^-1; c = e^T Omega e;
//   inlier iff m >= 0 and c <= c_max; log p -= inlier ? c : c_max;
//   inliers add J^T Omega J and J^T Omega e with J = d e / d xi (right
//   perturbation) to H and b.
//
// GB300 formulation (algebraically equal to the definition):
//  * Both covariances are GICP planes, Sigma = I - a n n^T (a = 1 - eps_cov),
//    so R Sigma^S R^T + Sigma^M = 2I - a (u u^T + w w^T) with u = R n_k,
//    w = n_m. With s = u + sg w, d = u - sg w (sg = sign(u.w)), s is orthogonal
//    to d and Omega = I/2 + a/(4 ls) s s^T + a/(4 ld) d d^T with
//    ls = 2 eps + (a/2)|d|^2, ld = 2 - (a/2)|d|^2: one reciprocal, no 3x3
//    inverse and no cancellation.
//  * J = R [ [mu]x , -I ] = [ [q~]x , -I ] diag(R, R), so the sums are taken in
//    the map frame with J~ = [ [q~]x , -I ] and rotated once per particle:
//    H = D H~ D^T, b = D b~ with D = diag(R^T, R^T).
//
// Layout: one thread per particle, particles visited in the order of the LSH
// sort (neighbouring poses share CTAs, so their NNF/map gathers share L1
// lines once the filter has converged); scan points stream through shared
// memory in 8 KB chunks, double-buffered with 1-D bulk copies (TMA,
// cp.async.bulk) completing on mbarriers; every thread of a warp reads the same
// point (broadcast). Accumulation in FP32 registers; the 29 sums are written as
// a structure of arrays in sorted order.
#include "mp_internal.cuh"

#include <cstdlib>

namespace {

constexpr int LK_THREADS = 128;
constexpr int LK_CHUNK = 256;   // points per stage: 256 x 32 B = 8 KB

struct LkArgs {
    const float4* poses;
    const int32_t* order;
    int64_t n;
    const float4* scan;
    const int32_t* nvalid;
    const int32_t* nnf;      // dense voxel grid of spatial-order map indices
    int nx, ny, nz;
    float inv_res, offx, offy, offz;
    const float4* rec;
    float c_max, half_a, two_eps, quarter_a;
    float* gn;
    int64_t stride;
    int32_t* err;
    unsigned long long* pairs;
    long long budget;   // cycle limit of each barrier wait
    int starve;         // test knob: announce 16 bytes more than copied for chunk 0
};

__device__ __forceinline__ void issue_chunk(const LkArgs& A, float4* dst, uint64_t* bar, int c, int nv) {
    int m = min(LK_CHUNK, nv - c * LK_CHUNK);
    uint32_t bytes = (uint32_t)m * 32u;
    mbar_expect_tx(bar, bytes + ((A.starve && c == 0) ? 16u : 0u));
    bulk_g2s(dst, A.scan + 2 * (int64_t)c * LK_CHUNK, bytes, bar);
}

// Sums of one particle over the scan (map frame, see the file comment).
struct LkAcc {
    float Hww[6];    // (00 01 02 11 12 22)
    float Hwv[9];    // row-major
    float Hvv[6];    // (00 01 02 11 12 22)
    float bw[3], bv[3];
    float ll;
    int cnt;
};

// Transformed point by the decision sequence.
__device__ __forceinline__ void lk_transform(const float R[9], float tx, float ty, float tz, const float4& P0,
                                             float& qtx, float& qty, float& qtz, float& qx, float& qy, float& qz) {
    qtx = __fmaf_rn(R[2], P0.z, __fmaf_rn(R[1], P0.y, __fmul_rn(R[0], P0.x)));
    qty = __fmaf_rn(R[5], P0.z, __fmaf_rn(R[4], P0.y, __fmul_rn(R[3], P0.x)));
    qtz = __fmaf_rn(R[8], P0.z, __fmaf_rn(R[7], P0.y, __fmul_rn(R[6], P0.x)));
    qx = __fadd_rn(qtx, tx);
    qy = __fadd_rn(qty, ty);
    qz = __fadd_rn(qtz, tz);
}

// Gather pipeline of one scan point: the lookup transforms it and loads its
// NNF entry (the map index), then the map record is loaded; the arithmetic
// consumes both.
struct LkLook {
    int m;        // map index (-1: outside the grid or no map point)
    float qx, qy, qz;
};

__device__ __forceinline__ LkLook lk_lookup(const LkArgs& A, const float R[9], float tx, float ty, float tz,
                                            const float4& P0) {
    float qtx, qty, qtz;
    LkLook L;
    lk_transform(R, tx, ty, tz, P0, qtx, qty, qtz, L.qx, L.qy, L.qz);
    const int vx = floor_to_int(__fmaf_rn(L.qx, A.inv_res, A.offx));
    const int vy = floor_to_int(__fmaf_rn(L.qy, A.inv_res, A.offy));
    const int vz = floor_to_int(__fmaf_rn(L.qz, A.inv_res, A.offz));
    const bool in = (unsigned)vx < (unsigned)A.nx && (unsigned)vy < (unsigned)A.ny && (unsigned)vz < (unsigned)A.nz;
    L.m = -1;
    if (in) L.m = __ldg(A.nnf + ((vz * A.ny + vy) * A.nx + vx));
    return L;
}

__device__ __forceinline__ LkLook lk_none() {
    LkLook L;
    L.m = -1;
    L.qx = L.qy = L.qz = 0.f;
    return L;
}

__device__ __forceinline__ void lk_record(const LkArgs& A, int mm, float4& r0, float4& r1) {
    r0 = make_float4(0.f, 0.f, 0.f, 0.f);
    r1 = r0;
    if (mm >= 0) {
        r0 = __ldg(A.rec + 2 * mm);
        r1 = __ldg(A.rec + 2 * mm + 1);
    }
}

// One (particle, point) pair: cost, inlier test, and the map-frame sums.
__device__ __forceinline__ void lk_accumulate(const LkArgs& A, LkAcc& S, const float R[9], float tx, float ty, float tz,
                                              const float4& P0, const float4& P1, const LkLook& L, const float4& r0,
                                              const float4& r1) {
    // lever arm q~ = R mu (value path: q - t differs from the decision
    // sequence's R mu only by the rounding of the sum)
    const int mm = L.m;
    const float qx = L.qx, qy = L.qy, qz = L.qz;
    const float qtx = qx - tx, qty = qy - ty, qtz = qz - tz;
    const float ex = r0.x - qx, ey = r0.y - qy, ez = r0.z - qz;
    const float ux = R[0] * P0.w + R[1] * P1.x + R[2] * P1.y;
    const float uy = R[3] * P0.w + R[4] * P1.x + R[5] * P1.y;
    const float uz = R[6] * P0.w + R[7] * P1.x + R[8] * P1.y;
    const float wx = r0.w, wy = r1.x, wz = r1.y;
    const float sg = copysignf(1.f, ux * wx + uy * wy + uz * wz);
    const float sx = fmaf(sg, wx, ux), sy = fmaf(sg, wy, uy), sz = fmaf(sg, wz, uz);
    const float dx = fmaf(-sg, wx, ux), dy = fmaf(-sg, wy, uy), dz = fmaf(-sg, wz, uz);
    const float dd = dx * dx + dy * dy + dz * dz;
    const float ls = fmaf(A.half_a, dd, A.two_eps);
    const float ld = fmaf(-A.half_a, dd, 2.f);
    const float rr = __fdividef(A.quarter_a, ls * ld);
    const float as = ld * rr, ad = ls * rr;
    const float se = sx * ex + sy * ey + sz * ez;
    const float de = dx * ex + dy * ey + dz * ez;
    const float ee = ex * ex + ey * ey + ez * ez;
    const float cost = fmaf(0.5f, ee, fmaf(as * se, se, ad * de * de));
    const bool inl = (mm >= 0) && (cost <= A.c_max);
    S.ll -= inl ? cost : A.c_max;
    S.cnt += inl ? 1 : 0;
    const float h = inl ? 0.5f : 0.f;
    const float Pw = inl ? as : 0.f, Qw = inl ? ad : 0.f;
    const float Psx = Pw * sx, Psy = Pw * sy, Psz = Pw * sz;
    const float Qdx = Qw * dx, Qdy = Qw * dy, Qdz = Qw * dz;
    const float Oxx = fmaf(Psx, sx, fmaf(Qdx, dx, h));
    const float Oyy = fmaf(Psy, sy, fmaf(Qdy, dy, h));
    const float Ozz = fmaf(Psz, sz, fmaf(Qdz, dz, h));
    const float Oxy = fmaf(Psx, sy, Qdx * dy);
    const float Oxz = fmaf(Psx, sz, Qdx * dz);
    const float Oyz = fmaf(Psy, sz, Qdy * dz);
    const float gx = Oxx * ex + Oxy * ey + Oxz * ez;
    const float gy = Oxy * ex + Oyy * ey + Oyz * ez;
    const float gz = Oxz * ex + Oyz * ey + Ozz * ez;
    // Pm = [q~]x Omega
    const float P00 = qty * Oxz - qtz * Oxy, P01 = qty * Oyz - qtz * Oyy, P02 = qty * Ozz - qtz * Oyz;
    const float P10 = qtz * Oxx - qtx * Oxz, P11 = qtz * Oxy - qtx * Oyz, P12 = qtz * Oxz - qtx * Ozz;
    const float P20 = qtx * Oxy - qty * Oxx, P21 = qtx * Oyy - qty * Oxy, P22 = qtx * Oyz - qty * Oxz;
    // H~_ww += Pm [q~]x^T ; H~_wv += Pm ; H~_vv += Omega
    S.Hww[0] += qty * P02 - qtz * P01;
    S.Hww[1] += qtz * P00 - qtx * P02;
    S.Hww[2] += qtx * P01 - qty * P00;
    S.Hww[3] += qtz * P10 - qtx * P12;
    S.Hww[4] += qtx * P11 - qty * P10;
    S.Hww[5] += qtx * P21 - qty * P20;
    S.Hwv[0] += P00; S.Hwv[1] += P01; S.Hwv[2] += P02;
    S.Hwv[3] += P10; S.Hwv[4] += P11; S.Hwv[5] += P12;
    S.Hwv[6] += P20; S.Hwv[7] += P21; S.Hwv[8] += P22;
    S.Hvv[0] += Oxx; S.Hvv[1] += Oxy; S.Hvv[2] += Oxz; S.Hvv[3] += Oyy; S.Hvv[4] += Oyz; S.Hvv[5] += Ozz;
    // b~ = [ g x q~ ; -g ]
    S.bw[0] += gy * qtz - gz * qty;
    S.bw[1] += gz * qtx - gx * qtz;
    S.bw[2] += gx * qty - gy * qtx;
    S.bv[0] -= gx; S.bv[1] -= gy; S.bv[2] -= gz;
}

// MINB: CTAs per SM the registers must allow.
template <int MINB>
__global__ void __launch_bounds__(LK_THREADS, MINB) k_likelihood(const LkArgs A) {
    __shared__ __align__(128) float4 buf[2][2 * LK_CHUNK];
    __shared__ __align__(8) uint64_t bar[2];

    const int64_t p = (int64_t)blockIdx.x * LK_THREADS + threadIdx.x;
    const bool active = p < A.n;
    const int64_t i = active ? A.order[p] : 0;
    Quat q;
    float t[3];
    load_pose(A.poses, i, q, t);
    float R[9];
    quat_rot_exact(q, R);

    const int nv = *A.nvalid;
    const int nchunks = (nv + LK_CHUNK - 1) / LK_CHUNK;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(A.pairs, (unsigned long long)A.n * (unsigned long long)nv);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (nchunks > 0) issue_chunk(A, buf[0], &bar[0], 0, nv);
        if (nchunks > 1) issue_chunk(A, buf[1], &bar[1], 1, nv);
    }

    LkAcc S;
#pragma unroll
    for (int k = 0; k < 6; ++k) { S.Hww[k] = 0.f; S.Hvv[k] = 0.f; }
#pragma unroll
    for (int k = 0; k < 9; ++k) S.Hwv[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) { S.bw[k] = 0.f; S.bv[k] = 0.f; }
    S.ll = 0.f;
    S.cnt = 0;

    const float tx = t[0], ty = t[1], tz = t[2];
    bool failed = false;
    int c = 0;
    for (; c < nchunks; ++c) {
        const int b = c & 1;
        const uint32_t parity = (uint32_t)((c >> 1) & 1);
        bool got = mbar_wait_bounded(&bar[b], parity, A.budget);
        if (__syncthreads_or(!got)) { failed = true; break; }
        const int m = min(LK_CHUNK, nv - c * LK_CHUNK);
        if (active) {
            const float4* P = buf[b];
            // software pipeline over the two dependent gathers (NNF entry, map
            // record): every iteration issues the NNF load of point k+2 and
            // the record load of point k+1 before the arithmetic of point k,
            // so each gather has a whole point of arithmetic (and the other
            // warps' work) to land in. Invariant at the loop head: sc = point
            // k (record loaded), sb = point k+1 (map index loaded).
            LkLook sb = lk_none(), sc = lk_lookup(A, R, tx, ty, tz, P[0]);
            float4 rc0, rc1;
            lk_record(A, sc.m, rc0, rc1);
            if (m > 1) sb = lk_lookup(A, R, tx, ty, tz, P[2]);
            for (int k = 0; k < m; ++k) {
                const LkLook nb = (k + 2 < m) ? lk_lookup(A, R, tx, ty, tz, P[2 * (k + 2)]) : lk_none();
                float4 n0, n1;
                lk_record(A, sb.m, n0, n1);
                lk_accumulate(A, S, R, tx, ty, tz, P[2 * k], P[2 * k + 1], sc, rc0, rc1);
                sc = sb;
                sb = nb;
                rc0 = n0;
                rc1 = n1;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && c + 2 < nchunks) issue_chunk(A, buf[b], &bar[b], c + 2, nv);
    }
    if (failed) {
        if (threadIdx.x == 0) {
            atomicOr(A.err, MP_ERR_WAIT);
            // drain the copies still in flight (bounded)
            for (int k = c; k < min(c + 2, nchunks); ++k)
                mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1), A.budget);
        }
        return;
    }
    if (!active) return;

    // rotate the sums back to the sensor frame: blocks M -> R^T M R
    float Hw[3][3] = {{S.Hww[0], S.Hww[1], S.Hww[2]}, {S.Hww[1], S.Hww[3], S.Hww[4]}, {S.Hww[2], S.Hww[4], S.Hww[5]}};
    float Hc[3][3] = {{S.Hwv[0], S.Hwv[1], S.Hwv[2]}, {S.Hwv[3], S.Hwv[4], S.Hwv[5]}, {S.Hwv[6], S.Hwv[7], S.Hwv[8]}};
    float Hv[3][3] = {{S.Hvv[0], S.Hvv[1], S.Hvv[2]}, {S.Hvv[1], S.Hvv[3], S.Hvv[4]}, {S.Hvv[2], S.Hvv[4], S.Hvv[5]}};
    float Ow[3][3], Oc[3][3], Ov[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
            float sw = 0.f, sc = 0.f, sv = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    float rr = R[3 * k + a] * R[3 * l + bb];
                    sw += rr * Hw[k][l];
                    sc += rr * Hc[k][l];
                    sv += rr * Hv[k][l];
                }
            Ow[a][bb] = sw; Oc[a][bb] = sc; Ov[a][bb] = sv;
        }
    float bwr[3], bvr[3];
    rot_apply_T(R, S.bw, bwr);
    rot_apply_T(R, S.bv, bvr);
    float out[MP_GN];
    // upper rows of the 6x6 [ [Hww, Hwv], [Hwv^T, Hvv] ]
    int o = 0;
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int cc = r; cc < 6; ++cc) {
            float v;
            if (r < 3 && cc < 3) v = Ow[r][cc];
            else if (r < 3) v = Oc[r][cc - 3];
            else v = Ov[r - 3][cc - 3];
            out[o++] = v;
        }
    out[21] = bwr[0]; out[22] = bwr[1]; out[23] = bwr[2];
    out[24] = bvr[0]; out[25] = bvr[1]; out[26] = bvr[2];
    out[27] = S.ll;
    out[28] = (float)S.cnt;
#pragma unroll
    for (int f = 0; f < MP_GN; ++f) A.gn[(int64_t)f * A.stride + p] = out[f];
}

}  // namespace

int mp_launch_likelihood(mp_ctx* c) {
    LkArgs A;
    A.poses = c->poses[c->cur];
    A.order = c->sorted_ids;
    A.n = c->n;
    A.scan = c->scan_pts;
    A.nvalid = c->scan_nvalid;
    A.nnf = c->nnf;
    A.nx = c->nnf_dims[0]; A.ny = c->nnf_dims[1]; A.nz = c->nnf_dims[2];
    A.inv_res = c->nnf_inv_res;
    A.offx = c->nnf_off[0]; A.offy = c->nnf_off[1]; A.offz = c->nnf_off[2];
    A.rec = c->map_rec;
    float a = 1.f - c->p.eps_cov;
    A.c_max = c->p.c_max;
    A.half_a = 0.5f * a;
    A.two_eps = 2.f * c->p.eps_cov;
    A.quarter_a = 0.25f * a;
    A.gn = c->gn;
    A.stride = c->cap;
    A.err = c->dev_error;
    A.budget = c->wait_budget > 0 ? c->wait_budget : MP_WAIT_BUDGET;
    A.starve = c->starve_tx;
    A.pairs = c->pairs;
    // occupancy target of the kernel (MP_LK_VARIANT overrides the default for
    // tuning sweeps; every variant computes the same sums)
    static int variant = -1;
    if (variant < 0) {
        const char* env = getenv("MP_LK_VARIANT");
        variant = env ? atoi(env) : 0;
    }
    const unsigned grid = grid_for(c->n, LK_THREADS);
    switch (variant) {
        case 4: k_likelihood<4><<<grid, LK_THREADS, 0, c->stream>>>(A); break;
        case 5: k_likelihood<5><<<grid, LK_THREADS, 0, c->stream>>>(A); break;
        default: k_likelihood<6><<<grid, LK_THREADS, 0, c->stream>>>(A); break;
    }
    MP_LAUNCHED(c);
    return MP_OK;
}
