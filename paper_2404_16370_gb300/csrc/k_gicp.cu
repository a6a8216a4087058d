// Scan-to-scan GICP odometry of the prediction step (Sec. III-B): DeltaT_t
// ~ T_{t-1}^-1 T_t from the current scan (source) and the previous one
// (target), and Sigma^DeltaT from the Gauss-Newton Hessian at the result.
//
// One iteration for the current estimate T = (R, t) (FP64, in device memory):
//  * k_gicp_iter, one thread per source point: decisions in FP32 on T's
//    rounding to float (R from the unit quaternion, q = R mu + t by the fixed
//    sequence, squared distances un-fused); the correspondence is the valid
//    target point of smallest squared distance, ties to the smaller index,
//    within r_corr (brute force over the target in shared-memory tiles; the
//    scans have at most a few thousand points). Each correspondence adds
//    J^T Omega J and J^T Omega e with the GICP plane covariances (the same
//    closed-form Omega and target-frame sums as the likelihood kernel); the
//    CTA reduces its points and writes one partial.
//  * k_gicp_solve, one thread: sums the partials in FP64, rotates the
//    target-frame sums to the source frame, solves the damped system
//    (Gaussian elimination with partial pivoting) and sets T <- T exp(delta);
//    once max |delta| < tol the state is marked converged and the remaining
//    launched iterations return at once. The Hessian of the last iteration is
//    kept: Sigma^DeltaT = H^-1 is taken on the host.
#include "mp_internal.cuh"

#include <cmath>
#include <cstring>

struct GicpBufs {
    int cap;
    float *src_raw, *tgt_raw, *src_n, *tgt_n;
    uint8_t *src_v, *tgt_v;
    float4 *src4, *tgt4, *tmp4;
    float* partial;     // blocks x 32
    double* state;      // q[4], t[3], H[21], done flag, iterations, n_corr
    float* prev;        // previous scan kept for mp_step_gicp (cap x 3)
    int n_prev;
    double last_T[16];
    int have_last;
};

namespace {

constexpr int GB = 256;        // threads per CTA (source points)
constexpr int GTILE = 256;     // target points per shared-memory tile
constexpr int NPART = 32;      // floats per partial: 27 sums + count (+ pad)
constexpr int ST_Q = 0, ST_T = 4, ST_H = 7, ST_DONE = 28, ST_IT = 29, ST_NC = 30, ST_N = 32;

__device__ __forceinline__ void state_pose32(const double* st, float R[9], float t[3]) {
    double qx = st[ST_Q], qy = st[ST_Q + 1], qz = st[ST_Q + 2], qw = st[ST_Q + 3];
    const double inv = 1.0 / sqrt(qx * qx + qy * qy + qz * qz + qw * qw);
    Quat q{(float)(qx * inv), (float)(qy * inv), (float)(qz * inv), (float)(qw * inv)};
    quat_rot_exact(q, R);
    t[0] = (float)st[ST_T];
    t[1] = (float)st[ST_T + 1];
    t[2] = (float)st[ST_T + 2];
}

__global__ void __launch_bounds__(GB) k_gicp_iter(const float4* __restrict__ src, int ns, const float4* __restrict__ tgt,
                                                  int nt, const double* __restrict__ state, float r2, float half_a,
                                                  float two_eps, float quarter_a, float* __restrict__ partial) {
    __shared__ float4 tp[GTILE];
    __shared__ float4 tn[GTILE];
    __shared__ float red[GB / 32][NPART];
    if (state[ST_DONE] != 0.0) return;   // converged: uniform across the grid
    float R[9], t[3];
    state_pose32(state, R, t);
    const int k = blockIdx.x * GB + threadIdx.x;
    const bool have = k < ns && src[2 * k + 1].z != 0.f;
    float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
    if (k < ns) { s0 = src[2 * k]; s1 = src[2 * k + 1]; }
    // transformed source point by the decision sequence
    const float qtx = __fmaf_rn(R[2], s0.z, __fmaf_rn(R[1], s0.y, __fmul_rn(R[0], s0.x)));
    const float qty = __fmaf_rn(R[5], s0.z, __fmaf_rn(R[4], s0.y, __fmul_rn(R[3], s0.x)));
    const float qtz = __fmaf_rn(R[8], s0.z, __fmaf_rn(R[7], s0.y, __fmul_rn(R[6], s0.x)));
    const float qx = __fadd_rn(qtx, t[0]), qy = __fadd_rn(qty, t[1]), qz = __fadd_rn(qtz, t[2]);
    float best = INFINITY;
    int bj = -1;
    float4 b0 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = b0;
    for (int j0 = 0; j0 < nt; j0 += GTILE) {
        __syncthreads();
        for (int j = threadIdx.x; j < GTILE; j += GB) {
            if (j0 + j < nt) {
                tp[j] = tgt[2 * (j0 + j)];
                tn[j] = tgt[2 * (j0 + j) + 1];
            }
        }
        __syncthreads();
        const int m = min(GTILE, nt - j0);
        if (have) {
            for (int j = 0; j < m; ++j) {
                if (tn[j].z == 0.f) continue;
                const float dx = __fsub_rn(tp[j].x, qx), dy = __fsub_rn(tp[j].y, qy), dz = __fsub_rn(tp[j].z, qz);
                const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                if (d2 < best) {
                    best = d2;
                    bj = j0 + j;
                    b0 = tp[j];
                    b1 = tn[j];
                }
            }
        }
    }
    float acc[NPART];
#pragma unroll
    for (int a = 0; a < NPART; ++a) acc[a] = 0.f;
    if (have && bj >= 0 && best <= r2) {
        // target-frame sums (J~ = [ [q~]x , -I ]), Omega in closed form
        const float ex = b0.x - qx, ey = b0.y - qy, ez = b0.z - qz;
        const float nsx = s0.w, nsy = s1.x, nsz = s1.y;      // source normal
        const float wx = b0.w, wy = b1.x, wz = b1.y;         // target normal
        const float ux = R[0] * nsx + R[1] * nsy + R[2] * nsz;
        const float uy = R[3] * nsx + R[4] * nsy + R[5] * nsz;
        const float uz = R[6] * nsx + R[7] * nsy + R[8] * nsz;
        const float sg = copysignf(1.f, ux * wx + uy * wy + uz * wz);
        const float sx = fmaf(sg, wx, ux), sy = fmaf(sg, wy, uy), sz = fmaf(sg, wz, uz);
        const float dx = fmaf(-sg, wx, ux), dy = fmaf(-sg, wy, uy), dz = fmaf(-sg, wz, uz);
        const float dd = dx * dx + dy * dy + dz * dz;
        const float ls = fmaf(half_a, dd, two_eps), ld = fmaf(-half_a, dd, 2.f);
        const float rr = quarter_a / (ls * ld);
        const float as = ld * rr, ad = ls * rr;
        const float Psx = as * sx, Psy = as * sy, Psz = as * sz, Qdx = ad * dx, Qdy = ad * dy, Qdz = ad * dz;
        const float Oxx = fmaf(Psx, sx, fmaf(Qdx, dx, 0.5f)), Oyy = fmaf(Psy, sy, fmaf(Qdy, dy, 0.5f));
        const float Ozz = fmaf(Psz, sz, fmaf(Qdz, dz, 0.5f));
        const float Oxy = fmaf(Psx, sy, Qdx * dy), Oxz = fmaf(Psx, sz, Qdx * dz), Oyz = fmaf(Psy, sz, Qdy * dz);
        const float gx = Oxx * ex + Oxy * ey + Oxz * ez;
        const float gy = Oxy * ex + Oyy * ey + Oyz * ez;
        const float gz = Oxz * ex + Oyz * ey + Ozz * ez;
        const float P00 = qty * Oxz - qtz * Oxy, P01 = qty * Oyz - qtz * Oyy, P02 = qty * Ozz - qtz * Oyz;
        const float P10 = qtz * Oxx - qtx * Oxz, P11 = qtz * Oxy - qtx * Oyz, P12 = qtz * Oxz - qtx * Ozz;
        const float P20 = qtx * Oxy - qty * Oxx, P21 = qtx * Oyy - qty * Oxy, P22 = qtx * Oyz - qty * Oxz;
        // Hww (6), Hwv (9), Hvv (6), bw (3), bv (3), count
        acc[0] = qty * P02 - qtz * P01;
        acc[1] = qtz * P00 - qtx * P02;
        acc[2] = qtx * P01 - qty * P00;
        acc[3] = qtz * P10 - qtx * P12;
        acc[4] = qtx * P11 - qty * P10;
        acc[5] = qtx * P21 - qty * P20;
        acc[6] = P00; acc[7] = P01; acc[8] = P02; acc[9] = P10; acc[10] = P11; acc[11] = P12;
        acc[12] = P20; acc[13] = P21; acc[14] = P22;
        acc[15] = Oxx; acc[16] = Oxy; acc[17] = Oxz; acc[18] = Oyy; acc[19] = Oyz; acc[20] = Ozz;
        acc[21] = gy * qtz - gz * qty;
        acc[22] = gz * qtx - gx * qtz;
        acc[23] = gx * qty - gy * qtx;
        acc[24] = -gx; acc[25] = -gy; acc[26] = -gz;
        acc[27] = 1.f;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 28; ++a) {
        const float v = warp_sum(acc[a]);
        if (lane == 0) red[w][a] = v;
    }
    __syncthreads();
    if (threadIdx.x < 28) {
        float v = 0.f;
        for (int q = 0; q < GB / 32; ++q) v += red[q][threadIdx.x];
        partial[blockIdx.x * NPART + threadIdx.x] = v;
    }
}

// FP64 SE(3) exp (rotation first), quaternion (x, y, z, w) and translation
__device__ void se3_exp_d(const double xi[6], double q[4], double t[3]) {
    const double wx = xi[0], wy = xi[1], wz = xi[2];
    const double th2 = wx * wx + wy * wy + wz * wz, th = sqrt(th2);
    double s, c, a, b;   // sin(th/2)/th, cos(th/2), (1-cos th)/th^2, (th-sin th)/th^3
    if (th < 1e-4) {
        s = 0.5 - th2 / 48.0;
        c = 1.0 - th2 / 8.0;
        a = 0.5 - th2 / 24.0;
        b = 1.0 / 6.0 - th2 / 120.0;
    } else {
        s = sin(0.5 * th) / th;
        c = cos(0.5 * th);
        a = (1.0 - cos(th)) / th2;
        b = (th - sin(th)) / (th2 * th);
    }
    q[0] = s * wx; q[1] = s * wy; q[2] = s * wz; q[3] = c;
    const double v[3] = {xi[3], xi[4], xi[5]};
    const double wv[3] = {wy * v[2] - wz * v[1], wz * v[0] - wx * v[2], wx * v[1] - wy * v[0]};
    const double wwv[3] = {wy * wv[2] - wz * wv[1], wz * wv[0] - wx * wv[2], wx * wv[1] - wy * wv[0]};
    for (int k = 0; k < 3; ++k) t[k] = v[k] + a * wv[k] + b * wwv[k];
}

__device__ void quat_R_d(const double q[4], double R[9]) {
    const double x = q[0], y = q[1], z = q[2], w = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

__global__ void k_gicp_solve(const float* __restrict__ partial, int nblocks, double* __restrict__ st, double lambda,
                             double eps, double tol) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    if (st[ST_DONE] != 0.0) return;
    double S[28];
    for (int a = 0; a < 28; ++a) S[a] = 0.0;
    for (int bI = 0; bI < nblocks; ++bI)
        for (int a = 0; a < 28; ++a) S[a] += (double)partial[bI * NPART + a];
    // rotate the target-frame blocks to the source frame: M -> R^T M R
    double qn[4] = {st[ST_Q], st[ST_Q + 1], st[ST_Q + 2], st[ST_Q + 3]};
    const double inv = 1.0 / sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
    for (int k = 0; k < 4; ++k) qn[k] *= inv;
    double R[9];
    quat_R_d(qn, R);
    const int sym[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    double Hw[3][3], Hc[3][3], Hv[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            Hw[r][c] = S[sym[r][c]];
            Hc[r][c] = S[6 + 3 * r + c];
            Hv[r][c] = S[15 + sym[r][c]];
        }
    double A[6][7];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            double w_ = 0, x_ = 0, v_ = 0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    const double rr = R[3 * k + a] * R[3 * l + c];
                    w_ += rr * Hw[k][l];
                    x_ += rr * Hc[k][l];
                    v_ += rr * Hv[k][l];
                }
            A[a][c] = w_;
            A[a][3 + c] = x_;
            A[3 + c][a] = x_;
            A[3 + a][3 + c] = v_;
        }
    double bvec[6];
    for (int a = 0; a < 3; ++a) {
        bvec[a] = R[a] * S[21] + R[3 + a] * S[22] + R[6 + a] * S[23];
        bvec[3 + a] = R[a] * S[24] + R[3 + a] * S[25] + R[6 + a] * S[26];
    }
    int o = 0;
    for (int r = 0; r < 6; ++r)
        for (int c = r; c < 6; ++c) st[ST_H + o++] = A[r][c];
    st[ST_NC] = S[27];
    st[ST_IT] += 1.0;
    for (int r = 0; r < 6; ++r) {
        A[r][r] += lambda * A[r][r] + eps;
        A[r][6] = -bvec[r];
    }
    bool ok = S[27] >= 6.0;
    for (int c = 0; c < 6 && ok; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (!(fabs(A[piv][c]) > 0.0)) { ok = false; break; }
        if (piv != c)
            for (int k = 0; k < 7; ++k) { double tmp = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = tmp; }
        for (int r = c + 1; r < 6; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int k = c; k < 7; ++k) A[r][k] -= f * A[c][k];
        }
    }
    if (!ok) { st[ST_DONE] = 2.0; return; }   // too few correspondences or singular
    double d[6];
    for (int r = 5; r >= 0; --r) {
        double v = A[r][6];
        for (int k = r + 1; k < 6; ++k) v -= A[r][k] * d[k];
        d[r] = v / A[r][r];
    }
    // T <- T exp(d)
    double dq[4], dt[3];
    se3_exp_d(d, dq, dt);
    double Rt[3];
    for (int r = 0; r < 3; ++r) Rt[r] = R[3 * r] * dt[0] + R[3 * r + 1] * dt[1] + R[3 * r + 2] * dt[2];
    const double ax = qn[0], ay = qn[1], az = qn[2], aw = qn[3];
    double nq[4] = {aw * dq[0] + ax * dq[3] + ay * dq[2] - az * dq[1], aw * dq[1] - ax * dq[2] + ay * dq[3] + az * dq[0],
                    aw * dq[2] + ax * dq[1] - ay * dq[0] + az * dq[3], aw * dq[3] - ax * dq[0] - ay * dq[1] - az * dq[2]};
    const double ni = 1.0 / sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
    for (int k = 0; k < 4; ++k) st[ST_Q + k] = nq[k] * ni;
    for (int k = 0; k < 3; ++k) st[ST_T + k] += Rt[k];
    double mx = 0.0;
    for (int k = 0; k < 6; ++k) mx = fmax(mx, fabs(d[k]));
    if (mx < tol) st[ST_DONE] = 1.0;
}

// packs n points (raw x 3, normals x 3, validity) into 2 float4: (mu, n.x), (n.y, n.z, valid, 0)
__global__ void k_gicp_pack(const float* __restrict__ raw, const float* __restrict__ nrm, const uint8_t* __restrict__ v,
                            int n, float4* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[2 * i] = make_float4(raw[3 * i], raw[3 * i + 1], raw[3 * i + 2], nrm[3 * i]);
    out[2 * i + 1] = make_float4(nrm[3 * i + 1], nrm[3 * i + 2], v[i] ? 1.f : 0.f, 0.f);
}

template <typename T>
cudaError_t galloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count > 0 ? count : 1));
}

int gicp_alloc(mp_ctx* c) {
    if (c->gicp) return MP_OK;
    GicpBufs* g = new GicpBufs();
    memset(g, 0, sizeof(*g));
    const int cap = c->p.max_scan;
    g->cap = cap;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t n) {
        if (e == cudaSuccess) e = galloc(p, n);
    };
    A(&g->src_raw, 3 * (size_t)cap); A(&g->tgt_raw, 3 * (size_t)cap); A(&g->src_n, 3 * (size_t)cap);
    A(&g->tgt_n, 3 * (size_t)cap); A(&g->src_v, cap); A(&g->tgt_v, cap); A(&g->src4, 2 * (size_t)cap);
    A(&g->tgt4, 2 * (size_t)cap); A(&g->tmp4, cap); A(&g->partial, (size_t)NPART * ((cap + GB - 1) / GB));
    A(&g->state, ST_N); A(&g->prev, 3 * (size_t)cap);
    c->gicp = g;
    if (e != cudaSuccess) return mp_cuda_check(c, e, "GICP buffers");
    return MP_OK;
}

// 6x6 SPD inverse on the host (Gauss-Jordan, FP64); false if singular
bool inv6(const double H[36], double I[36]) {
    double M[6][12];
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 12; ++c) M[r][c] = c < 6 ? H[6 * r + c] : (c - 6 == r ? 1.0 : 0.0);
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
        if (!(std::fabs(M[piv][c]) > 0.0)) return false;
        if (piv != c)
            for (int k = 0; k < 12; ++k) std::swap(M[c][k], M[piv][k]);
        const double d = M[c][c];
        for (int k = 0; k < 12; ++k) M[c][k] /= d;
        for (int r = 0; r < 6; ++r) {
            if (r == c) continue;
            const double f = M[r][c];
            for (int k = 0; k < 12; ++k) M[r][k] -= f * M[c][k];
        }
    }
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) I[6 * r + c] = M[r][6 + c];
    return true;
}

}  // namespace

void mp_gicp_free(mp_ctx* c) {
    GicpBufs* g = c->gicp;
    if (!g) return;
    void* bufs[] = {g->src_raw, g->tgt_raw, g->src_n, g->tgt_n, g->src_v, g->tgt_v, g->src4, g->tgt4, g->tmp4,
                    g->partial, g->state, g->prev};
    for (void* p : bufs)
        if (p) cudaFree(p);
    delete g;
    c->gicp = nullptr;
}

extern "C" {

int mp_gicp(mp_ctx* c, const float* src, int32_t n_src, const float* tgt, int32_t n_tgt, const double init_T[16],
            int32_t max_iters, double T_out[16], double cov_out[36], int32_t* n_corr, int32_t* iters) {
    if (!c) return MP_EINVAL;
    if (n_src < 1 || n_tgt < 1 || n_src > c->p.max_scan || n_tgt > c->p.max_scan || !src || !tgt || !T_out ||
        max_iters < 1)
        return mp_fail(c, MP_EINVAL, "mp_gicp: scans of 1..max_scan points, T_out and max_iters >= 1 required");
    int rc;
    if ((rc = gicp_alloc(c))) return rc;
    GicpBufs* g = c->gicp;
    MP_CUDA(c, cudaMemcpyAsync(g->src_raw, src, sizeof(float) * 3 * (size_t)n_src, cudaMemcpyDefault, c->stream));
    MP_CUDA(c, cudaMemcpyAsync(g->tgt_raw, tgt, sizeof(float) * 3 * (size_t)n_tgt, cudaMemcpyDefault, c->stream));
    if ((rc = mp_launch_point_gaussians(c, g->src_raw, n_src, g->tmp4, g->src_n, g->src_v))) return rc;
    k_gicp_pack<<<grid_for(n_src, 256), 256, 0, c->stream>>>(g->src_raw, g->src_n, g->src_v, n_src, g->src4);
    MP_LAUNCHED(c);
    if ((rc = mp_launch_point_gaussians(c, g->tgt_raw, n_tgt, g->tmp4, g->tgt_n, g->tgt_v))) return rc;
    k_gicp_pack<<<grid_for(n_tgt, 256), 256, 0, c->stream>>>(g->tgt_raw, g->tgt_n, g->tgt_v, n_tgt, g->tgt4);
    MP_LAUNCHED(c);
    // initial state from init_T (identity when NULL)
    double st[ST_N];
    memset(st, 0, sizeof(st));
    double q[4], t[3];
    odom_to_pose_host(init_T, q, t);
    for (int k = 0; k < 4; ++k) st[ST_Q + k] = q[k];
    for (int k = 0; k < 3; ++k) st[ST_T + k] = t[k];
    MP_CUDA(c, cudaMemcpyAsync(g->state, st, sizeof(st), cudaMemcpyHostToDevice, c->stream));
    const int nb = (n_src + GB - 1) / GB;
    const float a = 1.f - c->p.eps_cov;
    const float r2 = c->p.r_max * c->p.r_max;
    for (int it = 0; it < max_iters; ++it) {
        k_gicp_iter<<<nb, GB, 0, c->stream>>>(g->src4, n_src, g->tgt4, n_tgt, g->state, r2, 0.5f * a,
                                               2.f * c->p.eps_cov, 0.25f * a, g->partial);
        MP_LAUNCHED(c);
        k_gicp_solve<<<1, 32, 0, c->stream>>>(g->partial, nb, g->state, (double)c->p.lambda, (double)c->p.eps, 1e-6);
        MP_LAUNCHED(c);
    }
    MP_CUDA(c, cudaMemcpyAsync(st, g->state, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    MP_CUDA(c, cudaStreamSynchronize(c->stream));
    double R[9];
    const double nq = std::sqrt(st[0] * st[0] + st[1] * st[1] + st[2] * st[2] + st[3] * st[3]);
    const double x = st[0] / nq, y = st[1] / nq, z = st[2] / nq, w = st[3] / nq;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) T_out[4 * r + k] = R[3 * r + k];
        T_out[4 * r + 3] = st[ST_T + r];
    }
    T_out[12] = T_out[13] = T_out[14] = 0.0;
    T_out[15] = 1.0;
    if (n_corr) *n_corr = (int32_t)st[ST_NC];
    if (iters) *iters = (int32_t)st[ST_IT];
    if (st[ST_DONE] == 2.0) return mp_fail(c, MP_EINVAL, "mp_gicp: fewer than 6 correspondences or a singular system");
    if (cov_out) {
        double Hm[36];
        int o = 0;
        for (int r = 0; r < 6; ++r)
            for (int k = r; k < 6; ++k) {
                Hm[6 * r + k] = st[ST_H + o];
                Hm[6 * k + r] = st[ST_H + o];
                ++o;
            }
        if (!inv6(Hm, cov_out)) return mp_fail(c, MP_EINVAL, "mp_gicp: singular Hessian");
    }
    return MP_OK;
}

int mp_step_gicp(mp_ctx* c, const float* scan, int32_t n_scan, double cov_scale) {
    if (!c) return MP_EINVAL;
    if (c->n == 0) return mp_fail(c, MP_ENOTINIT, "particles not initialised");
    if (n_scan < 0 || n_scan > c->p.max_scan || (n_scan > 0 && !scan) || !(cov_scale >= 0.0))
        return mp_fail(c, MP_EINVAL, "mp_step_gicp: bad scan or cov_scale");
    int rc;
    if ((rc = gicp_alloc(c))) return rc;
    GicpBufs* g = c->gicp;
    if (n_scan == 0) {
        // blackout: no motion estimate; the next scan starts a new sequence
        g->n_prev = 0;
        g->have_last = 0;
        return mp_step(c, nullptr, 0, nullptr, nullptr);
    }
    double T[16], cov[36];
    if (g->n_prev > 0) {
        // constant-velocity start: the previous motion
        rc = mp_gicp(c, scan, n_scan, g->prev, g->n_prev, g->have_last ? g->last_T : nullptr, 30, T, cov, nullptr,
                     nullptr);
        if (rc) return rc;
        for (int k = 0; k < 36; ++k) cov[k] *= cov_scale;
        memcpy(g->last_T, T, sizeof(T));
        g->have_last = 1;
        if ((rc = mp_step(c, scan, n_scan, T, cov))) return rc;
    } else {
        if ((rc = mp_step(c, scan, n_scan, nullptr, nullptr))) return rc;
    }
    MP_CUDA(c, cudaMemcpyAsync(g->prev, scan, sizeof(float) * 3 * (size_t)n_scan, cudaMemcpyDefault, c->stream));
    g->n_prev = n_scan;
    return MP_OK;
}

}  // extern "C"
