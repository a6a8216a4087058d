// C ABI of the MegaParticles GB300 library (include/megaparticles.h): context
// lifecycle, the order of the stages of one filter step (Sec. III-B..III-D),
// host-side draws of T^LSH and delta^LSH (Eq. 10) and of nothing else, and
// buffer access for tests and state import/export.
#include "mp_internal.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <new>
#include <vector>

// Message of the last failure, on this thread, of a call that had no context
// to keep it (a failed mp_init_map, a batch, the allocation-free posterior,
// the proposal network): mp_last_error(NULL) returns it. The library prints
// nothing.
static thread_local char g_noctx_err[512];

int mp_fail(mp_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int mp_fail_noctx(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_noctx_err, sizeof(g_noctx_err), fmt, ap);
    va_end(ap);
    return code;
}

int mp_cuda_check(mp_ctx* c, cudaError_t e, const char* what) {
    int code = (e == cudaErrorMemoryAllocation) ? MP_ENOMEM : MP_ECUDA;
    return mp_fail(c, code, "%s: %s", what, cudaGetErrorString(e));
}

#ifdef MP_CHECKED
int mp_checked_sync(mp_ctx* c, const char* file, int line) {
    // MP_CHECKED_SYNC=0 keeps the device checks but not the synchronisation
    static const int sync = [] {
        const char* v = getenv("MP_CHECKED_SYNC");
        return v && v[0] == '0' ? 0 : 1;
    }();
    if (!sync) return MP_OK;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) return MP_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        fprintf(stderr, "MP_CHECKED: kernel launched at %s:%d: %s\n", file, line, cudaGetErrorString(e));
        return mp_fail(c, MP_ECUDA, "kernel launched at %s:%d: %s", file, line, cudaGetErrorString(e));
    }
    return MP_OK;
}
#endif

namespace {

// ---- host Philox-4x32-10 (Salmon et al., SC 2011) for the per-step LSH draw
void philox_host(const uint32_t in[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
    uint32_t x0 = in[0], x1 = in[1], x2 = in[2], x3 = in[3];
    for (int r = 0; r < 10; ++r) {
        uint64_t a = 0xD2511F53ull * x0, b = 0xCD9E8D57ull * x2;
        uint32_t y0 = (uint32_t)(b >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)b;
        uint32_t y2 = (uint32_t)(a >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// k-th 53-bit uniform of (seed, step, stream): words (2(k%2), 2(k%2)+1) of
// counter (k/2, 0, step, stream).
double u53_host(uint64_t seed, uint64_t step, uint32_t stream, uint32_t k) {
    uint32_t ctr[4] = {k >> 1, 0u, (uint32_t)step, stream}, o[4];
    philox_host(ctr, (uint32_t)seed, (uint32_t)(seed >> 32), o);
    uint32_t hi = o[(k & 1u) * 2], lo = o[(k & 1u) * 2 + 1];
    return (double)((((uint64_t)(hi >> 5)) << 26) | (uint64_t)(lo >> 6)) * (1.0 / 9007199254740992.0);
}

}  // namespace

// LSH draw of step c->step (Eq. 10): uniform rotation (Shoemake), translation
// uniform in the valid-map box, delta ~ N(0, lsh_sigma^2 I); host FP64 from
// Philox(seed, counter (k / 2, 0, step, LSH stream)).
void draw_lsh(mp_ctx* c) {
    double u[12];
    for (uint32_t k = 0; k < 12; ++k) u[k] = u53_host(c->p.seed, c->step, MP_STREAM_LSH, k);
    const double tau = 6.283185307179586476925286766559;
    double r1 = std::sqrt(1.0 - u[0]), r2 = std::sqrt(u[0]);
    c->lsh_q[0] = r1 * std::sin(tau * u[1]);
    c->lsh_q[1] = r1 * std::cos(tau * u[1]);
    c->lsh_q[2] = r2 * std::sin(tau * u[2]);
    c->lsh_q[3] = r2 * std::cos(tau * u[2]);
    for (int a = 0; a < 3; ++a) c->lsh_t[a] = c->map_lo[a] + u[3 + a] * (c->map_hi[a] - c->map_lo[a]);
    for (int k = 0; k < 3; ++k) {
        double rad = std::sqrt(-2.0 * std::log(1.0 - u[6 + 2 * k]));
        double ang = tau * u[7 + 2 * k];
        c->lsh_delta[2 * k] = (double)c->p.lsh_sigma * rad * std::cos(ang);
        c->lsh_delta[2 * k + 1] = (double)c->p.lsh_sigma * rad * std::sin(ang);
    }
}

// Per-step values of the current state (c->step, the LSH draw, the odometry)
// into a host StepDev; T_LSH is inverted here, in FP64.
void fill_step_host(mp_ctx* c, StepDev* h) {
    const double qx = c->lsh_q[0], qy = c->lsh_q[1], qz = c->lsh_q[2], qw = c->lsh_q[3];
    h->lsh_qinv[0] = -qx; h->lsh_qinv[1] = -qy; h->lsh_qinv[2] = -qz; h->lsh_qinv[3] = qw;
    double R[9];
    R[0] = 1 - 2 * (qy * qy + qz * qz); R[1] = 2 * (qx * qy - qw * qz); R[2] = 2 * (qx * qz + qw * qy);
    R[3] = 2 * (qx * qy + qw * qz); R[4] = 1 - 2 * (qx * qx + qz * qz); R[5] = 2 * (qy * qz - qw * qx);
    R[6] = 2 * (qx * qz - qw * qy); R[7] = 2 * (qy * qz + qw * qx); R[8] = 1 - 2 * (qx * qx + qy * qy);
    for (int r = 0; r < 3; ++r)
        h->lsh_tinv[r] = -(R[r] * c->lsh_t[0] + R[3 + r] * c->lsh_t[1] + R[6 + r] * c->lsh_t[2]);
    // rotation of the inverse quaternion: R^T
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) h->lsh_R[3 * r + k] = R[3 * k + r];
    for (int k = 0; k < 6; ++k) h->lsh_delta[k] = c->lsh_delta[k];
    for (int k = 0; k < 4; ++k) h->dq[k] = c->odom_q[k];
    for (int k = 0; k < 3; ++k) h->dt[k] = c->odom_t[k];
    for (int k = 0; k < 21; ++k) h->L[k] = c->chol[k];
    h->noise = c->noise;
    h->step = (uint32_t)c->step;
}

// Copies the per-step values to the device on the context stream: from the
// batch's fixed slot when one is set, else from the next slot of the pinned
// ring (waiting, if needed, until the copy that last used it has run).
int upload_step(mp_ctx* c) {
    StepDev* h = c->batch_slot;
    int slot = -1;
    if (!h) {
        slot = c->step_ring;
        c->step_ring ^= 1;
        MP_CUDA(c, cudaEventSynchronize(c->step_ev[slot]));
        h = c->step_host + slot;
    }
    fill_step_host(c, h);
    MP_CUDA(c, cudaMemcpyAsync(c->step_dev, h, sizeof(StepDev), cudaMemcpyHostToDevice, c->stream));
    if (slot >= 0) MP_CUDA(c, cudaEventRecord(c->step_ev[slot], c->stream));
    return MP_OK;
}

namespace {

template <typename T>
int dalloc(mp_ctx* c, T** p, size_t count) {
    if (*p) return MP_OK;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
    if (e != cudaSuccess) return mp_cuda_check(c, e, "cudaMalloc");
    return MP_OK;
}

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void free_particles(mp_ctx* c) {
    dfree(c->poses[0]); dfree(c->poses[1]);
    dfree(c->logprior); dfree(c->post); dfree(c->post_tmp); dfree(c->post_init); dfree(c->post_invden); dfree(c->post_w);
    dfree(c->post_ids);
    dfree(c->loglik); dfree(c->n_in); dfree(c->keys); dfree(c->buckets); dfree(c->sorted_ids); dfree(c->rank); dfree(c->visit);
    dfree(c->seg); dfree(c->sort_keys[0]); dfree(c->sort_keys[1]); dfree(c->sort_ids[0]); dfree(c->sort_ids[1]);
    dfree(c->radix_counts); dfree(c->scan_tmp);
    dfree(c->nbr_ids[0]); dfree(c->nbr_ids[1]); dfree(c->nbr_k); dfree(c->nbr_d);
    dfree(c->gn); dfree(c->psi); dfree(c->pinv); dfree(c->phi); dfree(c->red);
    c->cap = 0;
    c->n = 0;
}

size_t scan_need(int64_t n) {
    size_t need = 0;
    while (n > 1) {
        n = (n + 4095) / 4096;
        need += (size_t)n;
    }
    return need + 1;
}

int alloc_particles(mp_ctx* c, int64_t n) {
    free_particles(c);
    int64_t K = c->p.K;
    int64_t nb = (n + MP_SORT_TILE - 1) / MP_SORT_TILE;
    int rc = 0;
#define A_(ptr, cnt) if ((rc = dalloc(c, &(ptr), (size_t)(cnt)))) return rc
    A_(c->poses[0], 2 * n);
    A_(c->logprior, n); A_(c->post, n); A_(c->post_tmp, n); A_(c->post_init, n); A_(c->post_invden, n); A_(c->post_w, n * K);
    A_(c->post_ids, n * K);
    A_(c->loglik, n); A_(c->n_in, n); A_(c->keys, n); A_(c->buckets, n); A_(c->sorted_ids, n); A_(c->rank, n); A_(c->visit, n);
    A_(c->seg, 2 * ((int64_t)1 << c->p.n_buckets_log2));
    A_(c->sort_keys[0], n); A_(c->sort_keys[1], n); A_(c->sort_ids[0], n); A_(c->sort_ids[1], n);
    A_(c->radix_counts, MP_RADIX * nb);
    c->scan_tmp_cap = scan_need(MP_RADIX * nb) + 64;
    A_(c->scan_tmp, c->scan_tmp_cap);
    A_(c->nbr_ids[0], n * K); A_(c->nbr_ids[1], n * K); A_(c->nbr_k, n * K); A_(c->nbr_d, n * K * 6);
    A_(c->gn, (int64_t)MP_GN * n); A_(c->psi, 8 * n); A_(c->phi, 8 * n);
    if (c->p.svgd_precond) A_(c->pinv, 24 * n);
    A_(c->red, 3 * (n / 256 + 2));
#undef A_
    c->cap = n;
    c->cur = 0;
    return MP_OK;
}

void destroy(mp_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_particles(c);
    // the map buffers go with the last context that uses them
    if (c->map_refs && c->map_refs->fetch_sub(1) > 1) {
        c->map_pts = nullptr; c->map_normals = nullptr; c->map_valid = nullptr; c->map_rec = nullptr;
        c->map_perm = nullptr; c->nnf = nullptr;
    } else {
        delete c->map_refs;
        dfree(c->map_pts); dfree(c->map_normals); dfree(c->map_valid); dfree(c->map_rec); dfree(c->map_perm);
        dfree(c->nnf);
    }
    c->map_refs = nullptr;
    dfree(c->scan_raw); dfree(c->scan_normals); dfree(c->scan_valid); dfree(c->scan_pair); dfree(c->scan_h2); dfree(c->scan_tmp4);
    dfree(c->scan_nvalid);
    dfree(c->scalars); dfree(c->best_idx); dfree(c->best_pose); dfree(c->dev_error); dfree(c->post_bar); dfree(c->pairs);
    dfree(c->step_dev);
    mp_gicp_free(c);
    if (c->step_host) cudaFreeHost(c->step_host);
    for (int k = 0; k < 2; ++k)
        if (c->step_ev[k]) cudaEventDestroy(c->step_ev[k]);
    for (int r = 0; r < MP_EV_RING; ++r)
        for (int s = 0; s < MP_NSTAGES; ++s)
            for (int k = 0; k < 2; ++k)
                if (c->ev[r][s][k]) cudaEventDestroy(c->ev[r][s][k]);
    free(c->host_tmp);
    delete c;
}

int check_params(mp_ctx* c, const mp_params* p) {
    if (!(p->nnf_res > 0) || !(p->r_max > 0) || !(p->c_max > 0) || !(p->r_cov > 0))
        return mp_fail(c, MP_EINVAL, "nnf_res, r_max, c_max and r_cov must be positive");
    if (!(p->sigma_r > 0) || !(p->sigma_t > 0)) return mp_fail(c, MP_EINVAL, "sigma_r and sigma_t must be positive");
    if (!(p->eps_cov > 0 && p->eps_cov < 1)) return mp_fail(c, MP_EINVAL, "eps_cov must lie in (0, 1)");
    if (!(p->lambda >= 0) || !(p->eps >= 0) || !(p->alpha >= 0) || !(p->lsh_sigma >= 0))
        return mp_fail(c, MP_EINVAL, "lambda, eps, alpha and lsh_sigma must be non-negative");
    if (p->K < 1 || p->K > MP_MAXK) return mp_fail(c, MP_EINVAL, "K must lie in [1, %d]", MP_MAXK);
    if (p->C < 0 || p->C > 32) return mp_fail(c, MP_EINVAL, "C must lie in [0, 32]");
    if (p->cov_k < 3 || p->cov_k > MP_COVK || p->cov_min < 3 || p->cov_min > p->cov_k)
        return mp_fail(c, MP_EINVAL, "need 3 <= cov_min <= cov_k <= %d", MP_COVK);
    if (p->post_iters < 0 || p->post_iters > 1000) return mp_fail(c, MP_EINVAL, "post_iters must lie in [0, 1000]");
    if (p->n_buckets_log2 < 1 || p->n_buckets_log2 > 26) return mp_fail(c, MP_EINVAL, "n_buckets_log2 must lie in [1, 26]");
    if (p->max_scan < 1 || p->max_scan > (1 << 20)) return mp_fail(c, MP_EINVAL, "max_scan must lie in [1, 2^20]");
    if (p->svgd_precond != 0 && p->svgd_precond != 1) return mp_fail(c, MP_EINVAL, "svgd_precond must be 0 or 1");
    if (!(p->post_floor >= 0.f && p->post_floor <= 700.f))
        return mp_fail(c, MP_EINVAL, "post_floor must lie in [0, 700] nats (0: no floor)");
    return MP_OK;
}

// Rotation part of a row-major 4x4 to a unit quaternion (largest-diagonal
// branch), translation from the last column.
void odom_to_pose(const double T[16], double q[4], double t[3]) {
    double m00 = T[0], m01 = T[1], m02 = T[2], m10 = T[4], m11 = T[5], m12 = T[6], m20 = T[8], m21 = T[9], m22 = T[10];
    double tr = m00 + m11 + m22;
    double w, x, y, z;
    if (tr > m00 && tr > m11 && tr > m22) {
        double r = std::sqrt(1.0 + tr);
        w = 0.5 * r; x = (m21 - m12) / (2 * r); y = (m02 - m20) / (2 * r); z = (m10 - m01) / (2 * r);
    } else if (m00 >= m11 && m00 >= m22) {
        double r = std::sqrt(1.0 + m00 - m11 - m22);
        x = 0.5 * r; w = (m21 - m12) / (2 * r); y = (m01 + m10) / (2 * r); z = (m02 + m20) / (2 * r);
    } else if (m11 >= m22) {
        double r = std::sqrt(1.0 + m11 - m00 - m22);
        y = 0.5 * r; w = (m02 - m20) / (2 * r); x = (m01 + m10) / (2 * r); z = (m12 + m21) / (2 * r);
    } else {
        double r = std::sqrt(1.0 + m22 - m00 - m11);
        z = 0.5 * r; w = (m10 - m01) / (2 * r); x = (m02 + m20) / (2 * r); y = (m12 + m21) / (2 * r);
    }
    double nrm = std::sqrt(w * w + x * x + y * y + z * z);
    q[0] = x / nrm; q[1] = y / nrm; q[2] = z / nrm; q[3] = w / nrm;
    t[0] = T[3]; t[1] = T[7]; t[2] = T[11];
}

}  // namespace

void odom_to_pose_host(const double T[16], double q[4], double t[3]) {
    if (!T) {
        q[0] = q[1] = q[2] = 0.0;
        q[3] = 1.0;
        t[0] = t[1] = t[2] = 0.0;
        return;
    }
    odom_to_pose(T, q, t);
}

namespace {

// Lower Cholesky factor of a symmetric PSD 6x6, column by column; a column
// whose pivot is not positive is left zero (no noise along it).
void chol6(const double S[36], double L[6][6]) {
    for (int r = 0; r < 6; ++r)
        for (int k = 0; k < 6; ++k) L[r][k] = 0.0;
    for (int k = 0; k < 6; ++k) {
        double piv = S[6 * k + k];
        for (int m = 0; m < k; ++m) piv -= L[k][m] * L[k][m];
        if (!(piv > 1e-300)) continue;
        double d = std::sqrt(piv);
        L[k][k] = d;
        for (int r = k + 1; r < 6; ++r) {
            double acc = S[6 * r + k];
            for (int m = 0; m < k; ++m) acc -= L[r][m] * L[k][m];
            L[r][k] = acc / d;
        }
    }
}

// a device scratch of `bytes` for layout conversions in getters/setters
struct DevTmp {
    void* p = nullptr;
    ~DevTmp() { if (p) cudaFree(p); }
};

// Stage timing: run r of stage s uses event pair ev[r % RING][s]; before a
// pair is reused its (long completed) interval is folded into the total.
int stage_begin(mp_ctx* c, int s) {
    if (!c->timing) return MP_OK;
    int64_t r = c->stage_runs[s];
    int slot = (int)(r % MP_EV_RING);
    if (r >= MP_EV_RING) {
        float ms = 0.f;
        MP_CUDA(c, cudaEventSynchronize(c->ev[slot][s][1]));
        MP_CUDA(c, cudaEventElapsedTime(&ms, c->ev[slot][s][0], c->ev[slot][s][1]));
        c->stage_ms[s] += ms;
    }
    MP_CUDA(c, cudaEventRecord(c->ev[slot][s][0], c->stream));
    return MP_OK;
}
int stage_end(mp_ctx* c, int s) {
    if (!c->timing) return MP_OK;
    int slot = (int)(c->stage_runs[s] % MP_EV_RING);
    MP_CUDA(c, cudaEventRecord(c->ev[slot][s][1], c->stream));
    c->stage_runs[s]++;
    return MP_OK;
}

}  // namespace

extern "C" {

int mp_default_params(mp_params* p, int preset, int64_t n_particles) {
    if (!p) return MP_EINVAL;
    memset(p, 0, sizeof(*p));
    p->c_max = 9.0f;
    p->sigma_r = 5.0f;
    p->sigma_t = 2.5f;
    p->alpha = 1.0f;
    p->lsh_sigma = 0.5f;
    p->lambda = 1e-3f;
    p->eps = 1e-6f;
    p->eps_cov = 1e-3f;
    p->cov_k = 10;
    p->cov_min = 5;
    p->post_iters = 10;
    p->max_scan = 16384;
    p->seed = 4;
    p->post_floor = 700.0f;
    if (preset == MP_PRESET_BOX_ROOM) {
        p->nnf_res = 0.1f; p->r_max = 1.0f; p->r_cov = 1.0f; p->K = 16; p->C = 16;
    } else if (preset == MP_PRESET_OUTDOOR) {
        p->nnf_res = 0.2f; p->r_max = 2.0f; p->r_cov = 2.0f; p->K = 32; p->C = 32;
    } else {
        return MP_EINVAL;
    }
    int lb = 1;
    while (((int64_t)1 << lb) < n_particles && lb < 26) ++lb;
    p->n_buckets_log2 = lb;
    return MP_OK;
}

const char* mp_last_error(const mp_ctx* ctx) { return ctx ? ctx->err : g_noctx_err; }

// Everything of a context but its map: scan buffers, step scalars, staging,
// events.
static int ctx_setup(mp_ctx* c) {
    int rc = MP_OK;
    do {
        int64_t ms = c->p.max_scan;
        if ((rc = dalloc(c, &c->scan_raw, 3 * ms))) break;
        if ((rc = dalloc(c, &c->scan_normals, 3 * ms))) break;
        if ((rc = dalloc(c, &c->scan_valid, ms))) break;
        if ((rc = dalloc(c, &c->scan_pair, 3 * ms))) break;
        if ((rc = dalloc(c, &c->scan_h2, 2 * ms))) break;
        if ((rc = dalloc(c, &c->scan_tmp4, ms))) break;
        if ((rc = dalloc(c, &c->scan_nvalid, 1))) break;
        if ((rc = dalloc(c, &c->scalars, 8))) break;
        if ((rc = dalloc(c, &c->best_idx, 1))) break;
        if ((rc = dalloc(c, &c->best_pose, 2))) break;
        if ((rc = dalloc(c, &c->dev_error, 1))) break;
        if ((rc = dalloc(c, &c->post_bar, 1))) break;
        if ((rc = dalloc(c, &c->step_dev, 1))) break;
        if ((rc = dalloc(c, &c->pairs, 1))) break;
        cudaError_t e = cudaHostAlloc((void**)&c->step_host, 2 * sizeof(StepDev), cudaHostAllocDefault);
        if (e != cudaSuccess) { rc = mp_cuda_check(c, e, "cudaHostAlloc"); break; }
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&c->step_ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) { rc = mp_cuda_check(c, e, "cudaEventCreate"); break; }
        e = cudaMemsetAsync(c->dev_error, 0, sizeof(int32_t), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->scan_nvalid, 0, sizeof(int32_t), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->pairs, 0, sizeof(unsigned long long), c->stream);
        if (e != cudaSuccess) { rc = mp_cuda_check(c, e, "memset"); break; }
        for (int r = 0; r < MP_EV_RING && !rc; ++r)
            for (int s = 0; s < MP_NSTAGES && !rc; ++s)
                for (int k = 0; k < 2 && !rc; ++k) {
                    e = cudaEventCreate(&c->ev[r][s][k]);
                    if (e != cudaSuccess) rc = mp_cuda_check(c, e, "event");
                }
    } while (0);
    c->odom_q[3] = 1.f;
    return rc;
}

int mp_init_map(mp_ctx** out, const float* xyz, int64_t n_map, const mp_params* p, void* cuda_stream) {
    if (!out) return mp_fail_noctx(MP_EINVAL, "mp_init_map: NULL ctx pointer");
    *out = nullptr;
    mp_ctx* c = new (std::nothrow) mp_ctx();
    if (!c) return mp_fail_noctx(MP_ENOMEM, "mp_init_map: out of host memory");
    memset((void*)c, 0, sizeof(*c));
    int rc = MP_OK;
    if (!xyz || n_map <= 0 || !p) {
        destroy(c);
        return mp_fail_noctx(MP_EINVAL, "mp_init_map: empty map or NULL argument");
    }
    if (n_map >= ((int64_t)1 << 31)) {
        destroy(c);
        return mp_fail_noctx(MP_EINVAL, "mp_init_map: %lld map points (at most 2^31 - 1)", (long long)n_map);
    }
    if ((rc = check_params(c, p))) {
        mp_fail_noctx(rc, "mp_init_map: %s", c->err);
        destroy(c);
        return rc;
    }
    c->p = *p;
    c->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);
    c->n_map = n_map;
    c->map_refs = new (std::nothrow) std::atomic<int>(1);
    if (!c->map_refs) { destroy(c); return MP_ENOMEM; }
    float* xyz_dev = nullptr;
    do {
        if ((rc = dalloc(c, &c->map_pts, n_map))) break;
        if ((rc = dalloc(c, &c->map_normals, 3 * n_map))) break;
        if ((rc = dalloc(c, &c->map_valid, n_map))) break;
        if ((rc = dalloc(c, &c->map_rec, 2 * n_map))) break;
        if ((rc = ctx_setup(c))) break;
        if ((rc = dalloc(c, &xyz_dev, 3 * n_map))) break;
        cudaError_t e = cudaMemcpyAsync(xyz_dev, xyz, sizeof(float) * 3 * (size_t)n_map, cudaMemcpyDefault, c->stream);
        if (e != cudaSuccess) { rc = mp_cuda_check(c, e, "map upload"); break; }
        rc = mp_launch_map_prepare(c, xyz_dev);
        if (rc) break;
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) { rc = mp_cuda_check(c, e, "map preprocessing"); break; }
    } while (0);
    if (xyz_dev) cudaFree(xyz_dev);
    if (rc) {
        mp_fail_noctx(rc, "mp_init_map: %s", c->err);
        destroy(c);
        return rc;
    }
    *out = c;
    return MP_OK;
}

int mp_init_map_shared(mp_ctx** out, mp_ctx* src, const mp_params* p, void* cuda_stream) {
    if (!out) return mp_fail_noctx(MP_EINVAL, "mp_init_map_shared: NULL ctx pointer");
    *out = nullptr;
    if (!src || !p || !src->map_refs || src->n_map <= 0)
        return mp_fail_noctx(MP_EINVAL, "mp_init_map_shared: NULL argument or a source context without a map");
    mp_ctx* c = new (std::nothrow) mp_ctx();
    if (!c) return mp_fail_noctx(MP_ENOMEM, "mp_init_map_shared: out of host memory");
    memset((void*)c, 0, sizeof(*c));
    int rc = check_params(c, p);
    const mp_params& q = src->p;
    if (!rc && (p->nnf_res != q.nnf_res || p->r_max != q.r_max || p->r_cov != q.r_cov || p->cov_k != q.cov_k ||
                p->cov_min != q.cov_min))
        rc = mp_fail(c, MP_EINVAL, "mp_init_map_shared: nnf_res, r_max, r_cov, cov_k and cov_min must equal the "
                                   "source context's (they define the map)");
    cudaGetDevice(&c->device);
    if (!rc && c->device != src->device)
        rc = mp_fail(c, MP_EINVAL, "mp_init_map_shared: the source context belongs to device %d, not %d", src->device,
                     c->device);
    if (rc) {
        mp_fail_noctx(rc, "%s", c->err);
        destroy(c);
        return rc;
    }
    c->p = *p;
    c->stream = (cudaStream_t)cuda_stream;
    // the map: the source's device buffers (read only from here on) and its geometry
    c->n_map = src->n_map;
    c->n_map_valid = src->n_map_valid;
    c->map_pts = src->map_pts;
    c->map_normals = src->map_normals;
    c->map_valid = src->map_valid;
    c->map_rec = src->map_rec;
    c->map_perm = src->map_perm;
    c->nnf = src->nnf;
    memcpy(c->nnf_dims, src->nnf_dims, sizeof(c->nnf_dims));
    c->nnf_voxels = src->nnf_voxels;
    memcpy(c->nnf_origin, src->nnf_origin, sizeof(c->nnf_origin));
    c->nnf_inv_res = src->nnf_inv_res;
    memcpy(c->nnf_off, src->nnf_off, sizeof(c->nnf_off));
    memcpy(c->map_lo, src->map_lo, sizeof(c->map_lo));
    memcpy(c->map_hi, src->map_hi, sizeof(c->map_hi));
    src->map_refs->fetch_add(1);
    c->map_refs = src->map_refs;
    if ((rc = ctx_setup(c))) {
        mp_fail_noctx(rc, "mp_init_map_shared: %s", c->err);
        destroy(c);
        return rc;
    }
    // the source's map preprocessing ran on its own stream
    cudaError_t e = cudaStreamSynchronize(src->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        rc = mp_cuda_check(c, e, "mp_init_map_shared");
        mp_fail_noctx(rc, "%s", c->err);
        destroy(c);
        return rc;
    }
    *out = c;
    return MP_OK;
}

int mp_init_particles(mp_ctx* c, int64_t n, const float lo[6], const float hi[6], const float* poses,
                      const double* log_prior) {
    if (!c) return MP_EINVAL;
    if (n <= 0 || n > ((int64_t)1 << 26)) return mp_fail(c, MP_EINVAL, "n_particles must lie in [1, 2^26]");
    if (!poses && (!lo || !hi)) return mp_fail(c, MP_EINVAL, "need poses or bounds");
    MP_CUDA(c, cudaStreamSynchronize(c->stream));
    int rc = alloc_particles(c, n);
    if (rc) return rc;
    c->n = n;
    c->step = 0;
    if (poses) {
        float* tmp = nullptr;
        MP_CUDA(c, cudaMalloc(&tmp, sizeof(float) * 7 * (size_t)n));
        MP_CUDA(c, cudaMemcpyAsync(tmp, poses, sizeof(float) * 7 * (size_t)n, cudaMemcpyDefault, c->stream));
        rc = mp_launch_pack_poses(c, tmp, c->poses[0]);
        cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
        if (rc) return rc;
    } else {
        for (int a = 0; a < 6; ++a)
            if (!(hi[a] >= lo[a])) return mp_fail(c, MP_EINVAL, "bounds: hi < lo");
        if ((rc = mp_launch_init_uniform(c, lo, hi))) return rc;
    }
    if (log_prior) {
        MP_CUDA(c, cudaMemcpyAsync(c->logprior, log_prior, sizeof(double) * (size_t)n, cudaMemcpyDefault, c->stream));
    } else {
        MP_CUDA(c, cudaMemsetAsync(c->logprior, 0, sizeof(double) * (size_t)n, c->stream));
    }
    // lists = {self}, k = 1
    std::vector<int32_t> ids((size_t)(n * c->p.K), -1);
    std::vector<float> kk((size_t)(n * c->p.K), 0.f);
    for (int64_t i = 0; i < n; ++i) { ids[(size_t)(i * c->p.K)] = (int32_t)i; kk[(size_t)(i * c->p.K)] = 1.f; }
    c->nbr_cur = 0;
    MP_CUDA(c, cudaMemcpyAsync(c->nbr_ids[0], ids.data(), sizeof(int32_t) * ids.size(), cudaMemcpyHostToDevice, c->stream));
    MP_CUDA(c, cudaMemcpyAsync(c->nbr_k, kk.data(), sizeof(float) * kk.size(), cudaMemcpyHostToDevice, c->stream));
    MP_CUDA(c, cudaMemsetAsync(c->nbr_d, 0, sizeof(float) * 6 * ids.size(), c->stream));
    std::vector<int32_t> iota((size_t)n);
    for (int64_t i = 0; i < n; ++i) iota[(size_t)i] = (int32_t)i;
    MP_CUDA(c, cudaMemcpyAsync(c->sorted_ids, iota.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    MP_CUDA(c, cudaMemcpyAsync(c->rank, iota.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    MP_CUDA(c, cudaMemcpyAsync(c->visit, iota.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    MP_CUDA(c, cudaMemsetAsync(c->loglik, 0, sizeof(float) * (size_t)n, c->stream));
    MP_CUDA(c, cudaMemsetAsync(c->psi, 0, sizeof(float) * 8 * (size_t)n, c->stream));
    MP_CUDA(c, cudaMemsetAsync(c->phi, 0, sizeof(float) * 8 * (size_t)n, c->stream));
    MP_CUDA(c, cudaStreamSynchronize(c->stream));
    return MP_OK;
}

int mp_set_scan(mp_ctx* c, const float* scan, int32_t n_scan) {
    if (!c) return MP_EINVAL;
    if (n_scan < 0 || n_scan > c->p.max_scan) return mp_fail(c, MP_EINVAL, "n_scan %d outside [0, %d]", n_scan, c->p.max_scan);
    if (n_scan > 0 && !scan) return mp_fail(c, MP_EINVAL, "NULL scan");
    c->n_scan = n_scan;
    if (n_scan > 0)
        MP_CUDA(c, cudaMemcpyAsync(c->scan_raw, scan, sizeof(float) * 3 * (size_t)n_scan, cudaMemcpyDefault, c->stream));
    return MP_OK;
}

int mp_set_odometry(mp_ctx* c, const double odom_T[16], const double odom_cov[36]) {
    if (!c) return MP_EINVAL;
    double q[4] = {0, 0, 0, 1}, t[3] = {0, 0, 0};
    if (odom_T) {
        for (int k = 0; k < 16; ++k)
            if (!std::isfinite(odom_T[k])) return mp_fail(c, MP_EINVAL, "odometry is not finite");
        odom_to_pose(odom_T, q, t);
    }
    for (int k = 0; k < 4; ++k) c->odom_q[k] = (float)q[k];
    for (int k = 0; k < 3; ++k) c->odom_t[k] = (float)t[k];
    c->noise = 0;
    for (int k = 0; k < 21; ++k) c->chol[k] = 0.f;
    if (odom_cov) {
        double L[6][6];
        chol6(odom_cov, L);
        int o = 0;
        for (int r = 0; r < 6; ++r)
            for (int k = 0; k <= r; ++k) {
                c->chol[o++] = (float)L[r][k];
                if (L[r][k] != 0.0) c->noise = 1;
            }
    }
    return MP_OK;
}

int mp_set_step_index(mp_ctx* c, uint64_t step) {
    if (!c) return MP_EINVAL;
    c->step = step;
    return MP_OK;
}

int mp_run_stages(mp_ctx* c, uint32_t mask) {
    if (!c) return MP_EINVAL;
    if (c->n == 0) return mp_fail(c, MP_ENOTINIT, "particles not initialised");
    int rc = MP_OK;
    if (mask & (MP_STAGE_PREDICT | MP_STAGE_LSH)) {
        if (mask & MP_STAGE_LSH) draw_lsh(c);
        if ((rc = upload_step(c))) return rc;
    }
    for (int s = 0; s < MP_NSTAGES; ++s) {
        uint32_t bit = 1u << s;
        if (!(mask & bit)) continue;
        if ((rc = stage_begin(c, s))) return rc;
        switch (bit) {
            case MP_STAGE_PREDICT: rc = mp_launch_predict(c); break;
            case MP_STAGE_SCAN: rc = mp_launch_scan_prepare(c); break;
            case MP_STAGE_LSH: rc = mp_launch_lsh_keys(c); break;
            case MP_STAGE_SORT: rc = mp_launch_sort(c); break;
            case MP_STAGE_MERGE: rc = mp_launch_merge(c); break;
            case MP_STAGE_LIKELIHOOD: rc = mp_launch_likelihood(c); break;
            case MP_STAGE_SOLVE: rc = mp_launch_solve(c); break;
            case MP_STAGE_SVGD: rc = mp_launch_svgd(c); break;
            case MP_STAGE_POSTERIOR: rc = mp_launch_posterior(c); break;
        }
        if (rc) return rc;
        if ((rc = stage_end(c, s))) return rc;
    }
    return MP_OK;
}

int mp_step(mp_ctx* c, const float* scan, int32_t n_scan, const double odom_T[16], const double odom_cov[36]) {
    if (!c) return MP_EINVAL;
    if (c->n == 0) return mp_fail(c, MP_ENOTINIT, "particles not initialised");
    int rc;
    if ((rc = mp_set_scan(c, scan, n_scan))) return rc;
    if ((rc = mp_set_odometry(c, odom_T, odom_cov))) return rc;
    uint32_t mask = MP_STAGE_ALL;
    // no motion and no noise: T dT exp(0) = T, the stored poses stay bit-identical
    if (!c->noise && c->odom_q[0] == 0.f && c->odom_q[1] == 0.f && c->odom_q[2] == 0.f && c->odom_q[3] == 1.f &&
        c->odom_t[0] == 0.f && c->odom_t[1] == 0.f && c->odom_t[2] == 0.f)
        mask &= ~MP_STAGE_PREDICT;
    if (n_scan == 0) {
        // blackout: no correction; the posterior is smoothed with a zero log-likelihood
        mask &= MP_STAGE_PREDICT | MP_STAGE_LSH | MP_STAGE_SORT | MP_STAGE_MERGE | MP_STAGE_POSTERIOR;
        MP_CUDA(c, cudaMemsetAsync(c->loglik, 0, sizeof(float) * (size_t)c->n, c->stream));
        MP_CUDA(c, cudaMemsetAsync(c->scan_nvalid, 0, sizeof(int32_t), c->stream));
    }
    if ((rc = mp_run_stages(c, mask))) return rc;
    c->step++;
    return MP_OK;
}

int mp_get_posterior(mp_ctx* c, float* poses_out, double* prob_out, float best_pose[7], double* best_prob) {
    if (!c) return MP_EINVAL;
    if (c->n == 0) return mp_fail(c, MP_ENOTINIT, "particles not initialised");
    int32_t err = 0;
    MP_CUDA(c, cudaMemcpyAsync(&err, c->dev_error, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    if (best_pose || best_prob) {
        float4 bp[2];
        double sc[4];
        MP_CUDA(c, cudaMemcpyAsync(bp, c->best_pose, sizeof(bp), cudaMemcpyDeviceToHost, c->stream));
        MP_CUDA(c, cudaMemcpyAsync(sc, c->scalars, sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
        MP_CUDA(c, cudaStreamSynchronize(c->stream));
        if (best_pose) {
            best_pose[0] = bp[0].x; best_pose[1] = bp[0].y; best_pose[2] = bp[0].z; best_pose[3] = bp[0].w;
            best_pose[4] = bp[1].x; best_pose[5] = bp[1].y; best_pose[6] = bp[1].z;
        }
        if (best_prob) *best_prob = sc[3];
    }
    int rc;
    if (poses_out && (rc = mp_get_buffer(c, MP_BUF_POSES, poses_out, 7 * c->n))) return rc;
    if (prob_out && (rc = mp_get_buffer(c, MP_BUF_POST, prob_out, c->n))) return rc;
    MP_CUDA(c, cudaStreamSynchronize(c->stream));
    if (err) {
        cudaMemsetAsync(c->dev_error, 0, sizeof(int32_t), c->stream);
        return mp_fail(c, MP_ETIMEOUT, "a bounded device-side wait gave up (error bits 0x%x)", err);
    }
    return MP_OK;
}

int mp_destroy(mp_ctx* c) {
    destroy(c);
    return MP_OK;
}

int mp_buffer_size(mp_ctx* c, int which, int64_t* count) {
    if (!c || !count) return MP_EINVAL;
    int64_t n = c->n, K = c->p.K;
    switch (which) {
        case MP_BUF_POSES: *count = 7 * n; break;
        case MP_BUF_LOG_PRIOR: case MP_BUF_KEYS: case MP_BUF_BUCKETS: case MP_BUF_SORTED_IDS: case MP_BUF_POST:
        case MP_BUF_VISIT_ORDER:
        case MP_BUF_POST_INIT: case MP_BUF_LOGLIK: *count = n; break;
        case MP_BUF_SEGMENTS: *count = 2 * n; break;
        case MP_BUF_NBR_IDS: case MP_BUF_NBR_K: *count = n * K; break;
        case MP_BUF_NBR_D: *count = n * K * 6; break;
        case MP_BUF_GN: *count = n * MP_GN; break;
        case MP_BUF_PSI: case MP_BUF_PHI: *count = 6 * n; break;
        case MP_BUF_SCAN_NORMALS: *count = 3 * (int64_t)c->n_scan; break;
        case MP_BUF_SCAN_VALID: *count = c->n_scan; break;
        case MP_BUF_MAP_NORMALS: *count = 3 * c->n_map; break;
        case MP_BUF_MAP_VALID: *count = c->n_map; break;
        case MP_BUF_LSH: *count = 13; break;
        default: return mp_fail(c, MP_EINVAL, "unknown buffer %d", which);
    }
    return MP_OK;
}

int mp_get_buffer(mp_ctx* c, int which, void* dst, int64_t count) {
    if (!c || !dst) return MP_EINVAL;
    int64_t want;
    int rc = mp_buffer_size(c, which, &want);
    if (rc) return rc;
    if (count != want) return mp_fail(c, MP_EINVAL, "buffer %d holds %lld elements, not %lld", which, (long long)want, (long long)count);
    if (count == 0) return MP_OK;
    int64_t n = c->n;
    auto copy = [&](const void* src, size_t bytes) -> int {
        MP_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
        MP_CUDA(c, cudaStreamSynchronize(c->stream));
        return MP_OK;
    };
    switch (which) {
        case MP_BUF_POSES: {
            DevTmp t;
            MP_CUDA(c, cudaMalloc(&t.p, sizeof(float) * 7 * (size_t)n));
            if ((rc = mp_launch_unpack_poses(c, c->poses[c->cur], (float*)t.p))) return rc;
            return copy(t.p, sizeof(float) * 7 * (size_t)n);
        }
        case MP_BUF_GN: {
            DevTmp t;
            MP_CUDA(c, cudaMalloc(&t.p, sizeof(float) * MP_GN * (size_t)n));
            if ((rc = mp_launch_gather_gn(c, (float*)t.p))) return rc;
            return copy(t.p, sizeof(float) * MP_GN * (size_t)n);
        }
        case MP_BUF_LOG_PRIOR: return copy(c->logprior, sizeof(double) * n);
        case MP_BUF_KEYS: return copy(c->keys, sizeof(uint32_t) * n);
        case MP_BUF_BUCKETS: return copy(c->buckets, sizeof(uint32_t) * n);
        case MP_BUF_SORTED_IDS: return copy(c->sorted_ids, sizeof(int32_t) * n);
        case MP_BUF_VISIT_ORDER: return copy(c->visit, sizeof(int32_t) * n);
        case MP_BUF_NBR_IDS: return copy(c->nbr_ids[c->nbr_cur], sizeof(int32_t) * n * c->p.K);
        case MP_BUF_NBR_K: return copy(c->nbr_k, sizeof(float) * n * c->p.K);
        case MP_BUF_NBR_D: return copy(c->nbr_d, sizeof(float) * n * c->p.K * 6);
        case MP_BUF_POST: return copy(c->post, sizeof(double) * n);
        case MP_BUF_LOGLIK: return copy(c->loglik, sizeof(float) * n);
        case MP_BUF_SCAN_NORMALS: return copy(c->scan_normals, sizeof(float) * 3 * (size_t)c->n_scan);
        case MP_BUF_SCAN_VALID: return copy(c->scan_valid, (size_t)c->n_scan);
        case MP_BUF_MAP_NORMALS: return copy(c->map_normals, sizeof(float) * 3 * (size_t)c->n_map);
        case MP_BUF_MAP_VALID: return copy(c->map_valid, (size_t)c->n_map);
        case MP_BUF_LSH: {
            double h[13];
            for (int k = 0; k < 4; ++k) h[k] = c->lsh_q[k];
            for (int k = 0; k < 3; ++k) h[4 + k] = c->lsh_t[k];
            for (int k = 0; k < 6; ++k) h[7 + k] = c->lsh_delta[k];
            MP_CUDA(c, cudaMemcpy(dst, h, sizeof(h), cudaMemcpyDefault));
            return MP_OK;
        }
        case MP_BUF_POST_INIT: {
            std::vector<double> h((size_t)n);
            double sc[4];
            MP_CUDA(c, cudaMemcpyAsync(h.data(), c->post_init, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
            MP_CUDA(c, cudaMemcpyAsync(sc, c->scalars, sizeof(sc), cudaMemcpyDeviceToHost, c->stream));
            MP_CUDA(c, cudaStreamSynchronize(c->stream));
            for (auto& v : h) v /= sc[1];
            MP_CUDA(c, cudaMemcpy(dst, h.data(), sizeof(double) * n, cudaMemcpyDefault));
            return MP_OK;
        }
        case MP_BUF_PSI: case MP_BUF_PHI: {
            std::vector<float> h((size_t)(8 * n)), o((size_t)(6 * n));
            MP_CUDA(c, cudaMemcpyAsync(h.data(), which == MP_BUF_PSI ? c->psi : c->phi, sizeof(float) * 8 * n,
                                       cudaMemcpyDeviceToHost, c->stream));
            MP_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int64_t i = 0; i < n; ++i)
                for (int a = 0; a < 6; ++a) o[(size_t)(6 * i + a)] = h[(size_t)(8 * i + a)];
            MP_CUDA(c, cudaMemcpy(dst, o.data(), sizeof(float) * 6 * n, cudaMemcpyDefault));
            return MP_OK;
        }
        case MP_BUF_SEGMENTS: {
            int64_t nbk = (int64_t)1 << c->p.n_buckets_log2;
            std::vector<uint32_t> b((size_t)n);
            std::vector<int32_t> seg((size_t)(2 * nbk)), o((size_t)(2 * n));
            MP_CUDA(c, cudaMemcpyAsync(b.data(), c->buckets, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, c->stream));
            MP_CUDA(c, cudaMemcpyAsync(seg.data(), c->seg, sizeof(int32_t) * 2 * nbk, cudaMemcpyDeviceToHost, c->stream));
            MP_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int64_t i = 0; i < n; ++i) {
                o[(size_t)(2 * i)] = seg[b[(size_t)i]];
                o[(size_t)(2 * i + 1)] = seg[(size_t)(nbk + b[(size_t)i])];
            }
            MP_CUDA(c, cudaMemcpy(dst, o.data(), sizeof(int32_t) * 2 * n, cudaMemcpyDefault));
            return MP_OK;
        }
    }
    return mp_fail(c, MP_EINVAL, "buffer %d is not readable", which);
}

int mp_set_buffer(mp_ctx* c, int which, const void* src, int64_t count) {
    if (!c || !src) return MP_EINVAL;
    int64_t want;
    int rc = mp_buffer_size(c, which, &want);
    if (rc) return rc;
    if (count != want) return mp_fail(c, MP_EINVAL, "buffer %d holds %lld elements, not %lld", which, (long long)want, (long long)count);
    int64_t n = c->n;
    auto put = [&](void* d, size_t bytes) -> int {
        MP_CUDA(c, cudaMemcpyAsync(d, src, bytes, cudaMemcpyDefault, c->stream));
        MP_CUDA(c, cudaStreamSynchronize(c->stream));
        return MP_OK;
    };
    switch (which) {
        case MP_BUF_POSES: {
            DevTmp t;
            MP_CUDA(c, cudaMalloc(&t.p, sizeof(float) * 7 * (size_t)n));
            MP_CUDA(c, cudaMemcpyAsync(t.p, src, sizeof(float) * 7 * (size_t)n, cudaMemcpyDefault, c->stream));
            if ((rc = mp_launch_pack_poses(c, (const float*)t.p, c->poses[c->cur]))) return rc;
            MP_CUDA(c, cudaStreamSynchronize(c->stream));
            return MP_OK;
        }
        case MP_BUF_LOG_PRIOR: return put(c->logprior, sizeof(double) * n);
        case MP_BUF_SORTED_IDS: case MP_BUF_VISIT_ORDER: case MP_BUF_NBR_IDS: {
            // kernels index particles by these entries: checked on the host first
            const bool perm = which != MP_BUF_NBR_IDS;
            const int64_t m = perm ? n : n * c->p.K;
            std::vector<int32_t> h((size_t)m);
            MP_CUDA(c, cudaStreamSynchronize(c->stream));
            MP_CUDA(c, cudaMemcpy(h.data(), src, sizeof(int32_t) * (size_t)m, cudaMemcpyDefault));
            if (perm) {
                std::vector<uint8_t> seen((size_t)n, 0);
                for (int32_t v : h) {
                    if (v < 0 || v >= n || seen[(size_t)v])
                        return mp_fail(c, MP_EINVAL, "%s must be a permutation of [0, n)",
                                       which == MP_BUF_SORTED_IDS ? "sorted ids" : "the visiting order");
                    seen[(size_t)v] = 1;
                }
            } else {
                for (int32_t v : h)
                    if (v < -1 || v >= n) return mp_fail(c, MP_EINVAL, "neighbour ids must lie in [-1, n)");
            }
            src = h.data();   // put() copies from src on the context stream
            void* dst = which == MP_BUF_SORTED_IDS ? (void*)c->sorted_ids
                        : which == MP_BUF_VISIT_ORDER ? (void*)c->visit : (void*)c->nbr_ids[c->nbr_cur];
            return put(dst, sizeof(int32_t) * (size_t)m);
        }
        case MP_BUF_NBR_K: return put(c->nbr_k, sizeof(float) * n * c->p.K);
        case MP_BUF_NBR_D: return put(c->nbr_d, sizeof(float) * n * c->p.K * 6);
        case MP_BUF_LOGLIK: return put(c->loglik, sizeof(float) * n);
        case MP_BUF_PSI: {
            std::vector<float> in((size_t)(6 * n)), h((size_t)(8 * n), 0.f);
            MP_CUDA(c, cudaMemcpy(in.data(), src, sizeof(float) * 6 * n, cudaMemcpyDefault));
            for (int64_t i = 0; i < n; ++i)
                for (int a = 0; a < 6; ++a) h[(size_t)(8 * i + a)] = in[(size_t)(6 * i + a)];
            MP_CUDA(c, cudaMemcpy(c->psi, h.data(), sizeof(float) * 8 * n, cudaMemcpyHostToDevice));
            return MP_OK;
        }
    }
    return mp_fail(c, MP_EINVAL, "buffer %d is not writable", which);
}

int mp_nnf_query(mp_ctx* c, const int32_t* vox, int64_t m, int32_t* out) {
    if (!c || (m > 0 && (!vox || !out))) return MP_EINVAL;
    if (m == 0) return MP_OK;
    DevTmp tv, to;
    MP_CUDA(c, cudaMalloc(&tv.p, sizeof(int32_t) * 3 * (size_t)m));
    MP_CUDA(c, cudaMalloc(&to.p, sizeof(int32_t) * (size_t)m));
    MP_CUDA(c, cudaMemcpyAsync(tv.p, vox, sizeof(int32_t) * 3 * (size_t)m, cudaMemcpyDefault, c->stream));
    int rc = mp_launch_nnf_query(c, (const int32_t*)tv.p, m, (int32_t*)to.p);
    if (rc) return rc;
    MP_CUDA(c, cudaMemcpyAsync(out, to.p, sizeof(int32_t) * (size_t)m, cudaMemcpyDefault, c->stream));
    MP_CUDA(c, cudaStreamSynchronize(c->stream));
    return MP_OK;
}

int mp_map_info(mp_ctx* c, float origin[3], int32_t dims[3], float* inv_res, float off[3], int64_t* n_valid) {
    if (!c) return MP_EINVAL;
    for (int a = 0; a < 3; ++a) {
        if (origin) origin[a] = c->nnf_origin[a];
        if (dims) dims[a] = c->nnf_dims[a];
        if (off) off[a] = c->nnf_off[a];
    }
    if (inv_res) *inv_res = c->nnf_inv_res;
    if (n_valid) *n_valid = c->n_map_valid;
    return MP_OK;
}

int mp_set_timing(mp_ctx* c, int enable) {
    if (!c) return MP_EINVAL;
    MP_CUDA(c, cudaStreamSynchronize(c->stream));
    c->timing = enable ? 1 : 0;
    if (enable) {
        for (int s = 0; s < MP_NSTAGES; ++s) {
            c->stage_runs[s] = 0;
            c->stage_ms[s] = 0.0;
        }
        MP_CUDA(c, cudaMemsetAsync(c->pairs, 0, sizeof(unsigned long long), c->stream));
    }
    return MP_OK;
}

int mp_stage_times(mp_ctx* c, float ms[9], int64_t runs[9], int64_t* pairs) {
    if (!c) return MP_EINVAL;
    MP_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int s = 0; s < MP_NSTAGES; ++s) {
        double tot = c->stage_ms[s];
        int64_t r = c->stage_runs[s];
        int64_t first = r > MP_EV_RING ? r - MP_EV_RING : 0;
        for (int64_t k = first; k < r; ++k) {
            float m = 0.f;
            int slot = (int)(k % MP_EV_RING);
            MP_CUDA(c, cudaEventElapsedTime(&m, c->ev[slot][s][0], c->ev[slot][s][1]));
            tot += m;
        }
        if (ms) ms[s] = (float)tot;
        if (runs) runs[s] = r;
    }
    if (pairs) {
        unsigned long long v = 0;
        MP_CUDA(c, cudaMemcpy(&v, c->pairs, sizeof(v), cudaMemcpyDeviceToHost));
        *pairs = (int64_t)v;
    }
    return MP_OK;
}

int mp_debug_set(mp_ctx* c, int what, int64_t value) {
    if (!c) return MP_EINVAL;
    switch (what) {
        case MP_DEBUG_WAIT_BUDGET: c->wait_budget = value > 0 ? (long long)value : 0; return MP_OK;
        case MP_DEBUG_STARVE_TX: c->starve_tx = value ? 1 : 0; return MP_OK;
        case MP_DEBUG_STARVE_BARRIER: c->starve_bar = value ? 1 : 0; return MP_OK;
    }
    return mp_fail(c, MP_EINVAL, "unknown debug knob %d", what);
}

int mp_set_likelihood_split(mp_ctx* c, int split) {
    if (!c) return MP_EINVAL;
    if (split < 1 || split > 64) return mp_fail(c, MP_EINVAL, "likelihood split %d outside [1, 64]", split);
    c->lk_split = split;
    return MP_OK;
}

int mp_set_precision(mp_ctx* c, int precision) {
    if (!c) return MP_EINVAL;
    if (precision != MP_PREC_FP32 && precision != MP_PREC_BF16 && precision != MP_PREC_FP16)
        return mp_fail(c, MP_EINVAL, "unknown precision %d", precision);
    c->precision = precision;
    return MP_OK;
}

int mp_kernel_launches(mp_ctx* c, int64_t* count) {
    if (!c || !count) return MP_EINVAL;
    *count = c->launches;
    return MP_OK;
}

}  // extern "C"
