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

namespace {

constexpr int LK_THREADS = 128;
constexpr int LK_CHUNK = 256;   // points per stage: 256 x 32 B = 8 KB

struct LkArgs {
    const float4* poses;
    const int32_t* order;
    int64_t n;
    const float4* scan;
    const int32_t* nvalid;
    const int32_t* nnf;
    int nx, ny, nz;
    float inv_res, offx, offy, offz;
    const float4* rec;
    float c_max, half_a, two_eps, quarter_a;
    float* gn;
    int64_t stride;
    int32_t* err;
    unsigned long long* pairs;
};

__device__ __forceinline__ void issue_chunk(const LkArgs& A, float4* dst, uint64_t* bar, int c, int nv) {
    int m = min(LK_CHUNK, nv - c * LK_CHUNK);
    uint32_t bytes = (uint32_t)m * 32u;
    mbar_expect_tx(bar, bytes);
    bulk_g2s(dst, A.scan + 2 * (int64_t)c * LK_CHUNK, bytes, bar);
}

__global__ void __launch_bounds__(LK_THREADS, 4) k_likelihood(const LkArgs A) {
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

    float Hww0 = 0, Hww1 = 0, Hww2 = 0, Hww3 = 0, Hww4 = 0, Hww5 = 0;     // (00 01 02 11 12 22)
    float Hwv00 = 0, Hwv01 = 0, Hwv02 = 0, Hwv10 = 0, Hwv11 = 0, Hwv12 = 0, Hwv20 = 0, Hwv21 = 0, Hwv22 = 0;
    float Hvv0 = 0, Hvv1 = 0, Hvv2 = 0, Hvv3 = 0, Hvv4 = 0, Hvv5 = 0;
    float bw0 = 0, bw1 = 0, bw2 = 0, bv0 = 0, bv1 = 0, bv2 = 0;
    float ll = 0.f;
    int cnt = 0;

    const float tx = t[0], ty = t[1], tz = t[2];
    bool failed = false;
    int c = 0;
    for (; c < nchunks; ++c) {
        const int b = c & 1;
        const uint32_t parity = (uint32_t)((c >> 1) & 1);
        bool got = mbar_wait_bounded(&bar[b], parity, MP_WAIT_BUDGET);
        if (__syncthreads_or(!got)) { failed = true; break; }
        const int m = min(LK_CHUNK, nv - c * LK_CHUNK);
        if (active) {
            const float4* P = buf[b];
#pragma unroll 4
            for (int k = 0; k < m; ++k) {
                const float4 P0 = P[2 * k], P1 = P[2 * k + 1];
                // transformed point by the decision sequence
                const float qtx = __fmaf_rn(R[2], P0.z, __fmaf_rn(R[1], P0.y, __fmul_rn(R[0], P0.x)));
                const float qty = __fmaf_rn(R[5], P0.z, __fmaf_rn(R[4], P0.y, __fmul_rn(R[3], P0.x)));
                const float qtz = __fmaf_rn(R[8], P0.z, __fmaf_rn(R[7], P0.y, __fmul_rn(R[6], P0.x)));
                const float qx = __fadd_rn(qtx, tx), qy = __fadd_rn(qty, ty), qz = __fadd_rn(qtz, tz);
                const int vx = floor_to_int(__fmaf_rn(qx, A.inv_res, A.offx));
                const int vy = floor_to_int(__fmaf_rn(qy, A.inv_res, A.offy));
                const int vz = floor_to_int(__fmaf_rn(qz, A.inv_res, A.offz));
                const bool in = (unsigned)vx < (unsigned)A.nx && (unsigned)vy < (unsigned)A.ny &&
                                (unsigned)vz < (unsigned)A.nz;
                int mm = -1;
                if (in) mm = __ldg(A.nnf + ((vz * A.ny + vy) * A.nx + vx));
                float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
                if (mm >= 0) {
                    r0 = __ldg(A.rec + 2 * mm);
                    r1 = __ldg(A.rec + 2 * mm + 1);
                }
                // residual and information matrix (map frame)
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
                ll -= inl ? cost : A.c_max;
                cnt += inl ? 1 : 0;
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
                Hww0 += qty * P02 - qtz * P01;
                Hww1 += qtz * P00 - qtx * P02;
                Hww2 += qtx * P01 - qty * P00;
                Hww3 += qtz * P10 - qtx * P12;
                Hww4 += qtx * P11 - qty * P10;
                Hww5 += qtx * P21 - qty * P20;
                Hwv00 += P00; Hwv01 += P01; Hwv02 += P02;
                Hwv10 += P10; Hwv11 += P11; Hwv12 += P12;
                Hwv20 += P20; Hwv21 += P21; Hwv22 += P22;
                Hvv0 += Oxx; Hvv1 += Oxy; Hvv2 += Oxz; Hvv3 += Oyy; Hvv4 += Oyz; Hvv5 += Ozz;
                // b~ = [ g x q~ ; -g ]
                bw0 += gy * qtz - gz * qty;
                bw1 += gz * qtx - gx * qtz;
                bw2 += gx * qty - gy * qtx;
                bv0 -= gx; bv1 -= gy; bv2 -= gz;
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
                mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1), MP_WAIT_BUDGET);
        }
        return;
    }
    if (!active) return;

    // rotate the sums back to the sensor frame: blocks M -> R^T M R
    float Hw[3][3] = {{Hww0, Hww1, Hww2}, {Hww1, Hww3, Hww4}, {Hww2, Hww4, Hww5}};
    float Hc[3][3] = {{Hwv00, Hwv01, Hwv02}, {Hwv10, Hwv11, Hwv12}, {Hwv20, Hwv21, Hwv22}};
    float Hv[3][3] = {{Hvv0, Hvv1, Hvv2}, {Hvv1, Hvv3, Hvv4}, {Hvv2, Hvv4, Hvv5}};
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
    const float bwm[3] = {bw0, bw1, bw2}, bvm[3] = {bv0, bv1, bv2};
    rot_apply_T(R, bwm, bwr);
    rot_apply_T(R, bvm, bvr);
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
    out[27] = ll;
    out[28] = (float)cnt;
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
    A.pairs = c->pairs;
    k_likelihood<<<grid_for(c->n, LK_THREADS), LK_THREADS, 0, c->stream>>>(A);
    MP_LAUNCHED(c);
    return MP_OK;
}
