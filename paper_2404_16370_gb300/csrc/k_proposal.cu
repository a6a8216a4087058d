// Learned proposal: box-room sensor simulator, PointNet-style mixture network
// (forward, backward, Adam) and mixture sampling. The C ABI and the network's
// definition are in include/mp_proposal.h.
//
// Layout: activations row-major [rows][channels] in FP32, rows = batch x
// points for the shared per-point layers and = batch for the head. Every
// dense layer of the FP32 form is one tiled GEMM (64 x 64 output tile per
// CTA, 16-deep K slices in shared memory, 4 x 4 outputs per thread) with the
// bias and ReLU fused into the store; weight gradients reduce over rows with
// split-K CTAs adding into the gradient by atomics. The BF16 form's forward
// pass through the per-point layers is one tensor-core kernel (k_pn_tc.cu).
// The backward pass through the per-point layers runs on the max-pooled rows
// only (k_pool_rows).
#include "mp_internal.cuh"
#include "../../include/mp_proposal.h"

#include <algorithm>
#include <cstdio>

#define MP_STREAM_SIM 4u
#define MP_STREAM_PN_INIT 5u
#define MP_STREAM_PN_SAMPLE 6u

namespace {

constexpr int C1 = 64, C2 = 128, C3 = 256, C4 = 256;
constexpr int NOUT = MP_PN_OUT, NCOMP = MP_PN_COMPONENTS;
constexpr float LOGSTD_LIM = 3.f;

// offsets of the parameter blocks in the flat array
constexpr int64_t OW1 = 0, OB1 = OW1 + 3 * C1, OW2 = OB1 + C1, OB2 = OW2 + (int64_t)C1 * C2, OW3 = OB2 + C2,
                  OB3 = OW3 + (int64_t)C2 * C3, OW4 = OB3 + C3, OB4 = OW4 + (int64_t)C3 * C4, OW5 = OB4 + C4,
                  OB5 = OW5 + (int64_t)C4 * NOUT, NPARAM = OB5 + NOUT;

__device__ __forceinline__ float2 normal2(uint32_t a, uint32_t b) {
    const float rad = sqrtf(-2.f * logf(u32_to_open01(a)));
    float s, c;
    sincospif(2.f * u32_to_open01(b), &s, &c);
    return make_float2(rad * c, rad * s);
}

// ---------------------------------------------------------------------------
// sensor simulator
__global__ void k_sim_box_room(const float* __restrict__ boxes, int n_boxes, float half, float height,
                               const float* __restrict__ poses, int64_t B, const float* __restrict__ dirs, int P,
                               float noise, uint2 key, float* __restrict__ out) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= B * P) return;
    const int64_t b = idx / P;
    const int r = (int)(idx % P);
    const float* pz = poses + b * 7;
    Quat q{pz[0], pz[1], pz[2], pz[3]};
    q = qnormalize(q);
    float R[9];
    quat_rot(q, R);
    const float dx = dirs[3 * r], dy = dirs[3 * r + 1], dz = dirs[3 * r + 2];
    const float ox = pz[4], oy = pz[5], oz = pz[6];
    const float wx = R[0] * dx + R[1] * dy + R[2] * dz;
    const float wy = R[3] * dx + R[4] * dy + R[5] * dz;
    const float wz = R[6] * dx + R[7] * dy + R[8] * dz;
    // room interior: the nearest wall ahead on each axis
    auto wall = [](float o, float d, float lo, float hi) {
        return d > 0.f ? (hi - o) / d : (d < 0.f ? (lo - o) / d : INFINITY);
    };
    float t = fminf(fminf(wall(ox, wx, -half, half), wall(oy, wy, -half, half)), wall(oz, wz, 0.f, height));
    // yawed boxes: slab test in each box's frame, hits in front of the origin
    for (int k = 0; k < n_boxes; ++k) {
        const float* bx = boxes + 7 * k;
        float sn, cs;
        sincosf(-bx[6], &sn, &cs);
        const float lx = ox - bx[0], ly = oy - bx[1];
        const float o3[3] = {cs * lx - sn * ly, sn * lx + cs * ly, oz};
        const float d3[3] = {cs * wx - sn * wy, sn * wx + cs * wy, wz};
        const float lo3[3] = {-0.5f * bx[3], -0.5f * bx[4], bx[2]};
        const float hi3[3] = {0.5f * bx[3], 0.5f * bx[4], bx[2] + bx[5]};
        float tmin = -INFINITY, tmax = INFINITY;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d3[a] != 0.f) {
                const float inv = 1.f / d3[a];
                const float t1 = (lo3[a] - o3[a]) * inv, t2 = (hi3[a] - o3[a]) * inv;
                tmin = fmaxf(tmin, fminf(t1, t2));
                tmax = fminf(tmax, fmaxf(t1, t2));
            } else if (o3[a] < lo3[a] || o3[a] > hi3[a]) {
                tmin = INFINITY;   // parallel to the slab and outside it
            }
        }
        if (tmax >= tmin && tmin > 1e-6f && tmin < t) t = tmin;
    }
    const uint4 u = philox4x32_10(make_uint4((uint32_t)r, (uint32_t)b, (uint32_t)(b >> 32), MP_STREAM_SIM), key);
    const float rng = t + noise * normal2(u.x, u.y).x;
    float* o = out + 3 * idx;
    o[0] = dx * rng;
    o[1] = dy * rng;
    o[2] = dz * rng;
}

// ---------------------------------------------------------------------------
// dense layers: C[M x N] (+)= op(A)[M x K] op(B)[K x N], op = transpose when
// TA / TB; A is [M][K] (or [K][M]), B is [K][N] (or [N][K]).
enum : int { EPI_BIAS = 1, EPI_RELU = 2, EPI_ATOMIC = 4 };
constexpr int GT = 64, GK = 16;

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_gemm(const float* __restrict__ A, const float* __restrict__ B,
                                              float* __restrict__ C, const float* __restrict__ bias, int M, int N,
                                              int K, int lda, int ldb, int ldc, int kchunk) {
    __shared__ float As[GK][GT + 4];
    __shared__ float Bs[GK][GT + 4];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += GK) {
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int mm = TA ? e % GT : e / GK, kk = TA ? e / GT : e % GK;
            const int m = m0 + mm, k = k0 + kk;
            float v = 0.f;
            if (m < M && k < ke) v = TA ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
            As[kk][mm] = v;
        }
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int nn = TB ? e / GK : e % GT, kk = TB ? e % GK : e / GT;
            const int n = n0 + nn, k = k0 + kk;
            float v = 0.f;
            if (n < N && k < ke) v = TB ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float v = acc[i][j];
            if (EPI & EPI_ATOMIC) {
                atomicAdd(C + (int64_t)m * ldc + n, v);
            } else {
                if (EPI & EPI_BIAS) v += bias[n];
                if (EPI & EPI_RELU) v = fmaxf(v, 0.f);
                C[(int64_t)m * ldc + n] = v;
            }
        }
    }
}

// column sums of X [rows x n] added into out (bias gradients)
__global__ void k_colsum(const float* __restrict__ X, int64_t rows, int n, int rows_per_cta, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_cta, r1 = min(rows, r0 + rows_per_cta);
    float s = 0.f;
    for (int64_t r = r0; r < r1; ++r) s += X[r * n + c];
    atomicAdd(out + c, s);
}

// dX = dH where H > 0 else 0 (ReLU backward, in place)
__global__ void k_relu_back(float* __restrict__ dH, const float* __restrict__ H, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && !(H[i] > 0.f)) dH[i] = 0.f;
}

__global__ void k_scale_points(const float* __restrict__ x, int64_t n, float inv, float* __restrict__ y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i] * inv;
}

// g[b][c] = max over points of h3[b][p][c]; index of the first maximum
__global__ void k_maxpool(const float* __restrict__ h3, int B, int P, float* __restrict__ g, int* __restrict__ gi) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (c >= C3 || b >= B) return;
    const float* base = h3 + (int64_t)b * P * C3 + c;
    float m = base[0];
    int mi = 0;
    for (int p = 1; p < P; ++p) {
        const float v = base[(int64_t)p * C3];
        if (v > m) { m = v; mi = p; }
    }
    g[b * C3 + c] = m;
    gi[b * C3 + c] = mi;
}

__global__ void k_pool_rows(const float* __restrict__ dg, const float* __restrict__ g, const int* __restrict__ gi,
                            const float* __restrict__ xs, const float* __restrict__ h1, const float* __restrict__ h2,
                            const float* __restrict__ W3, int B, int P, float* __restrict__ xc,
                            float* __restrict__ h1c, float* __restrict__ h2c, float* __restrict__ dh2c) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // r = b * 256 + c
    if (r >= (int64_t)B * C3) return;
    const int64_t b = r / C3;
    const int c = (int)(r % C3);
    const float d = g[r] > 0.f ? dg[r] : 0.f;
    const int64_t row = b * P + gi[r];
    for (int k = 0; k < 3; ++k) xc[r * 3 + k] = xs[row * 3 + k];
    for (int k = 0; k < C1; ++k) h1c[r * C1 + k] = h1[row * C1 + k];
    for (int i = 0; i < C2; ++i) {
        const float h = h2[row * C2 + i];
        h2c[r * C2 + i] = h;
        dh2c[r * C2 + i] = h > 0.f ? d * W3[i * C3 + c] : 0.f;
    }
}

// dW3[i][c] += sum_b dg[b][c] h2[b, gi[b][c], i] (pooled, gated) and db3[c]
__global__ void k_dw3(const float* __restrict__ dg, const float* __restrict__ g, const int* __restrict__ gi,
                      const float* __restrict__ h2, int B, int P, float* __restrict__ dW3, float* __restrict__ db3) {
    const int c = blockIdx.x;          // channel
    const int i = threadIdx.x;         // input channel (C2 threads)
    float acc = 0.f, bacc = 0.f;
    for (int b = 0; b < B; ++b) {
        const int64_t r = (int64_t)b * C3 + c;
        if (!(g[r] > 0.f)) continue;
        const float d = dg[r];
        acc = fmaf(d, h2[((int64_t)b * P + gi[r]) * C2 + i], acc);
        bacc += d;
    }
    dW3[i * C3 + c] += acc;
    if (i == 0) db3[c] += bacc;
}

__device__ __forceinline__ float wrap_pi(float a) {
    // into (-pi, pi]
    a = a - 6.283185307179586f * floorf(a * 0.15915494309189535f + 0.5f);
    return a <= -3.14159265358979f ? a + 6.283185307179586f : a;
}

// Mixture negative log-likelihood of each sample and its gradient w.r.t. o,
// scaled by 1/B (mean loss).
__global__ void k_mdn_loss(const float* __restrict__ o, const float* __restrict__ y, int B,
                           float* __restrict__ dO, float* __restrict__ loss) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float* ob = o + (int64_t)b * NOUT;
    float* db = dO + (int64_t)b * NOUT;
    float yy[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) yy[d] = y[b * 6 + d];
    // log pi = a - logsumexp(a)
    float amax = -INFINITY;
    for (int c = 0; c < NCOMP; ++c) amax = fmaxf(amax, ob[c]);
    float asum = 0.f;
    for (int c = 0; c < NCOMP; ++c) asum += expf(ob[c] - amax);
    const float lse_a = amax + logf(asum);
    float lj[NCOMP];
    float jmax = -INFINITY;
    const float half_log_2pi6 = 3.f * 1.8378770664093453f;
    for (int c = 0; c < NCOMP; ++c) {
        float s = 0.f;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            const float ls = LOGSTD_LIM * tanhf(ob[224 + 6 * c + d] / LOGSTD_LIM);
            float dl = yy[d] - ob[32 + 6 * c + d];
            if (d == 3) dl = wrap_pi(dl);
            const float z = dl * expf(-ls);
            s += -0.5f * z * z - ls;
        }
        lj[c] = ob[c] - lse_a + s - half_log_2pi6;
        jmax = fmaxf(jmax, lj[c]);
    }
    float jsum = 0.f;
    for (int c = 0; c < NCOMP; ++c) jsum += expf(lj[c] - jmax);
    const float L = -(jmax + logf(jsum));
    atomicAdd(loss, L / B);
    const float invB = 1.f / B;
    for (int c = 0; c < NCOMP; ++c) {
        const float r = expf(lj[c] + L);               // responsibility
        const float pi = expf(ob[c] - lse_a);
        db[c] = (pi - r) * invB;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            const float th = tanhf(ob[224 + 6 * c + d] / LOGSTD_LIM);
            const float ls = LOGSTD_LIM * th;
            float dl = yy[d] - ob[32 + 6 * c + d];
            if (d == 3) dl = wrap_pi(dl);
            const float iv = expf(-2.f * ls);
            db[32 + 6 * c + d] = -r * dl * iv * invB;
            db[224 + 6 * c + d] = r * (1.f - dl * dl * iv) * (1.f - th * th) * invB;
        }
    }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// He-normal weights (std sqrt(2 / fan_in)), zero biases, last layer N(0, 0.01^2)
__global__ void k_pn_init(float* __restrict__ p, uint2 key) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    float std = 0.f;
    if (i < OB1) std = sqrtf(2.f / 3.f);
    else if (i >= OW2 && i < OB2) std = sqrtf(2.f / C1);
    else if (i >= OW3 && i < OB3) std = sqrtf(2.f / C2);
    else if (i >= OW4 && i < OB4) std = sqrtf(2.f / C3);
    else if (i >= OW5 && i < OB5) std = 0.01f;
    const uint4 u = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, MP_STREAM_PN_INIT), key);
    p[i] = std * normal2(u.x, u.y).x;
}

__global__ void k_pn_sample(const float* __restrict__ mix, int64_t n, uint2 key, const float* __restrict__ scale,
                            const float* __restrict__ offset, float* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float amax = -INFINITY;
    for (int c = 0; c < NCOMP; ++c) amax = fmaxf(amax, mix[c]);
    float tot = 0.f;
    for (int c = 0; c < NCOMP; ++c) tot += expf(mix[c] - amax);
    const uint4 u0 = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, MP_STREAM_PN_SAMPLE), key);
    const uint4 u1 = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 1u, MP_STREAM_PN_SAMPLE), key);
    const float pick = u32_to_open01(u0.x) * tot;
    int comp = NCOMP - 1;
    float acc = 0.f;
    for (int c = 0; c < NCOMP; ++c) {
        acc += expf(mix[c] - amax);
        if (pick < acc) { comp = c; break; }
    }
    const float2 z0 = normal2(u0.y, u0.z), z1 = normal2(u0.w, u1.x), z2 = normal2(u1.y, u1.z);
    const float z[6] = {z0.x, z0.y, z1.x, z1.y, z2.x, z2.y};
    float v[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const float ls = LOGSTD_LIM * tanhf(mix[224 + 6 * comp + d] / LOGSTD_LIM);
        v[d] = (mix[32 + 6 * comp + d] + expf(ls) * z[d]) * scale[d] + offset[d];
    }
    v[3] = wrap_pi(v[3]);
    // rotation from Z-Y-X Euler angles (yaw, pitch, roll): Rz Ry Rx
    float sy, cy, sp, cp, sr, cr;
    sincosf(0.5f * v[3], &sy, &cy);
    sincosf(0.5f * v[4], &sp, &cp);
    sincosf(0.5f * v[5], &sr, &cr);
    float* o = out + 7 * i;
    o[0] = sr * cp * cy - cr * sp * sy;
    o[1] = cr * sp * cy + sr * cp * sy;
    o[2] = cr * cp * sy - sr * sp * cy;
    o[3] = cr * cp * cy + sr * sp * sy;
    o[4] = v[0];
    o[5] = v[1];
    o[6] = v[2];
}

template <typename T>
cudaError_t dmalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count > 0 ? count : 1));
}

}  // namespace

struct mp_pn {
    int P, Bmax;
    float in_scale;
    float* scale;    // device [6]
    float* offset;   // device [6]
    cudaStream_t stream;
    float *param, *grad, *am, *av;
    int64_t t;       // Adam step
    float *xs, *h1, *h2, *h3, *g, *h4, *o;
    int* gi;
    float *dO, *dh4, *dg;
    float *xc, *h1c, *h2c, *dh2c, *dh1c;   // compact rows (b, channel) of the backward pass
    uint2 key;
    int prec;          // MP_PREC_BF16: per-point layers on the tensor cores; MP_PREC_FP32: CUDA cores
    uint8_t* wimg;     // BF16 image of W2^T and W3^T for the tensor-core kernel
    int32_t* err;      // device error bits of the fused kernel
};

namespace {

int pn_fail(const char* what, cudaError_t e) {
    return mp_fail_noctx(e == cudaErrorMemoryAllocation ? MP_ENOMEM : MP_ECUDA, "mp_pn: %s: %s", what,
                         cudaGetErrorString(e));
}

#define PN_CUDA(x)                                   \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) return pn_fail(#x, e_); \
    } while (0)

template <bool TA, bool TB, int EPI>
void gemm(cudaStream_t s, const float* A, const float* B, float* C, const float* bias, int M, int N, int K, int lda,
          int ldb, int ldc, int splits = 1) {
    const int kchunk = ((K + splits - 1) / splits + GK - 1) / GK * GK;
    const int nz = (K + kchunk - 1) / kchunk;
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, nz);
    k_gemm<TA, TB, EPI><<<grid, 256, 0, s>>>(A, B, C, bias, M, N, K, lda, ldb, ldc, kchunk);
}

// split count for a weight gradient that reduces over `rows` rows: enough
// CTAs to fill the GPU (~4 per SM)
int splits_for(int64_t rows, int M, int N) {
    const int64_t tiles = (int64_t)((M + GT - 1) / GT) * ((N + GT - 1) / GT);
    int64_t s = (4 * 152 + tiles - 1) / tiles;
    s = std::min<int64_t>(s, std::max<int64_t>(1, rows / 256));
    return (int)std::max<int64_t>(1, s);
}

void colsum(cudaStream_t s, const float* X, int64_t rows, int n, float* out) {
    const int rpc = 512;
    dim3 grid((n + 127) / 128, (unsigned)((rows + rpc - 1) / rpc));
    k_colsum<<<grid, 128, 0, s>>>(X, rows, n, rpc, out);
}

// BF16 image of the per-point weights, refreshed after every parameter update
int pack_weights(mp_pn* net) {
    if (net->prec != MP_PREC_BF16) return MP_OK;
    return mp_pn_tc_pack(net->param + OW2, net->param + OW3, net->wimg, net->stream);
}

// train: keep the per-point activations h1, h2 for the backward pass
int forward(mp_pn* net, const float* scans, int B, bool train) {
    cudaStream_t s = net->stream;
    const int64_t rows = (int64_t)B * net->P;
    k_scale_points<<<grid_for(rows * 3, 256), 256, 0, s>>>(scans, rows * 3, 1.f / net->in_scale, net->xs);
    const float* W = net->param;
    if (net->prec == MP_PREC_BF16) {
        const int rc = mp_pn_tc_forward(net->xs, B, net->P, W + OW1, W + OB1, W + OB2, W + OB3, net->wimg, net->g,
                                        net->gi, train ? net->h1 : nullptr, train ? net->h2 : nullptr, net->err,
                                        MP_WAIT_BUDGET, s);
        if (rc) return mp_fail_noctx(rc, "mp_pn: tensor-core forward launch failed");
    } else {
        gemm<false, false, EPI_BIAS | EPI_RELU>(s, net->xs, W + OW1, net->h1, W + OB1, (int)rows, C1, 3, 3, C1, C1);
        gemm<false, false, EPI_BIAS | EPI_RELU>(s, net->h1, W + OW2, net->h2, W + OB2, (int)rows, C2, C1, C1, C2, C2);
        gemm<false, false, EPI_BIAS | EPI_RELU>(s, net->h2, W + OW3, net->h3, W + OB3, (int)rows, C3, C2, C2, C3, C3);
        k_maxpool<<<dim3(C3 / 128, B), 128, 0, s>>>(net->h3, B, net->P, net->g, net->gi);
    }
    gemm<false, false, EPI_BIAS | EPI_RELU>(s, net->g, W + OW4, net->h4, W + OB4, B, C4, C3, C3, C4, C4);
    gemm<false, false, EPI_BIAS>(s, net->h4, W + OW5, net->o, W + OB5, B, NOUT, C4, C4, NOUT, NOUT);
    PN_CUDA(cudaGetLastError());
    return MP_OK;
}

}  // namespace

extern "C" {

int mp_pn_sim_box_room(const float* boxes, int n_boxes, float half, float height, const float* poses, int64_t B,
                       const float* dirs, int P, float noise, uint64_t seed, float* out, void* cuda_stream) {
    if (n_boxes < 0 || B < 0 || P < 0 || (n_boxes > 0 && !boxes) || (B * P > 0 && (!poses || !dirs || !out)))
        return mp_fail_noctx(MP_EINVAL, "mp_pn_sim_box_room: invalid argument");
    if (B * P == 0) return MP_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    k_sim_box_room<<<grid_for(B * P, 256), 256, 0, s>>>(boxes, n_boxes, half, height, poses, B, dirs, P, noise, key,
                                                          out);
    PN_CUDA(cudaGetLastError());
    return MP_OK;
}

int mp_pn_create(mp_pn** netp, int n_points, int max_batch, float in_scale, const float scale[6],
                 const float offset[6], uint64_t seed, void* cuda_stream) {
    if (!netp || n_points < 1 || max_batch < 1 || !(in_scale > 0.f) || !scale || !offset) return mp_fail_noctx(MP_EINVAL, "mp_pn_create: invalid argument");
    if ((int64_t)n_points * max_batch * C3 >= ((int64_t)1 << 31)) return mp_fail_noctx(MP_EINVAL, "mp_pn_create: invalid argument");
    mp_pn* net = new mp_pn();
    net->P = n_points;
    net->Bmax = max_batch;
    net->in_scale = in_scale;
    net->stream = (cudaStream_t)cuda_stream;
    net->key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const int64_t rows = (int64_t)n_points * max_batch;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t n) {
        if (e == cudaSuccess) e = dmalloc(p, n);
    };
    A(&net->scale, 6); A(&net->offset, 6);
    A(&net->param, NPARAM); A(&net->grad, NPARAM); A(&net->am, NPARAM); A(&net->av, NPARAM);
    A(&net->xs, rows * 3); A(&net->h1, rows * C1); A(&net->h2, rows * C2); A(&net->h3, rows * C3);
    A(&net->g, (size_t)max_batch * C3); A(&net->gi, (size_t)max_batch * C3); A(&net->h4, (size_t)max_batch * C4);
    A(&net->o, (size_t)max_batch * NOUT); A(&net->dO, (size_t)max_batch * NOUT);
    A(&net->dh4, (size_t)max_batch * C4); A(&net->dg, (size_t)max_batch * C3);
    const int64_t rows_c = (int64_t)max_batch * C3;
    A(&net->xc, rows_c * 3); A(&net->h1c, rows_c * C1); A(&net->h2c, rows_c * C2); A(&net->dh2c, rows_c * C2);
    A(&net->dh1c, rows_c * C1);
    A(&net->wimg, mp_pn_tc_image_bytes()); A(&net->err, 1);
    if (e != cudaSuccess) {
        mp_pn_destroy(net);
        return pn_fail("allocation", e);
    }
    *netp = net;
    PN_CUDA(cudaMemcpyAsync(net->scale, scale, 6 * sizeof(float), cudaMemcpyDefault, net->stream));
    PN_CUDA(cudaMemcpyAsync(net->offset, offset, 6 * sizeof(float), cudaMemcpyDefault, net->stream));
    PN_CUDA(cudaMemsetAsync(net->am, 0, sizeof(float) * NPARAM, net->stream));
    PN_CUDA(cudaMemsetAsync(net->av, 0, sizeof(float) * NPARAM, net->stream));
    PN_CUDA(cudaMemsetAsync(net->grad, 0, sizeof(float) * NPARAM, net->stream));
    PN_CUDA(cudaMemsetAsync(net->err, 0, sizeof(int32_t), net->stream));
    k_pn_init<<<grid_for(NPARAM, 256), 256, 0, net->stream>>>(net->param, net->key);
    PN_CUDA(cudaGetLastError());
    net->prec = n_points % 128 == 0 ? MP_PREC_BF16 : MP_PREC_FP32;
    if (pack_weights(net)) return pn_fail("weight image", cudaGetLastError());
    PN_CUDA(cudaStreamSynchronize(net->stream));
    return MP_OK;
}

int mp_pn_destroy(mp_pn* net) {
    if (!net) return mp_fail_noctx(MP_EINVAL, "mp_pn_destroy: invalid argument");
    void* bufs[] = {net->scale, net->offset, net->param, net->grad, net->am, net->av, net->xs, net->h1,
                    net->h2, net->h3, net->g, net->gi, net->h4, net->o, net->dO, net->dh4, net->dg, net->xc,
                    net->h1c, net->h2c, net->dh2c, net->dh1c, net->wimg, net->err};
    for (void* p : bufs)
        if (p) cudaFree(p);
    delete net;
    return MP_OK;
}

int mp_pn_num_params(mp_pn* net, int64_t* n) {
    if (!net || !n) return mp_fail_noctx(MP_EINVAL, "mp_pn_num_params: invalid argument");
    *n = NPARAM;
    return MP_OK;
}

int mp_pn_get_params(mp_pn* net, float* out) {
    if (!net || !out) return mp_fail_noctx(MP_EINVAL, "mp_pn_get_params: invalid argument");
    PN_CUDA(cudaMemcpyAsync(out, net->param, sizeof(float) * NPARAM, cudaMemcpyDefault, net->stream));
    PN_CUDA(cudaStreamSynchronize(net->stream));
    return MP_OK;
}

int mp_pn_set_params(mp_pn* net, const float* in) {
    if (!net || !in) return mp_fail_noctx(MP_EINVAL, "mp_pn_set_params: invalid argument");
    PN_CUDA(cudaMemcpyAsync(net->param, in, sizeof(float) * NPARAM, cudaMemcpyDefault, net->stream));
    if (pack_weights(net)) return pn_fail("weight image", cudaGetLastError());
    PN_CUDA(cudaStreamSynchronize(net->stream));
    return MP_OK;
}

int mp_pn_forward(mp_pn* net, const float* scans, int B, float* out) {
    if (!net || !scans || !out || B < 1 || B > net->Bmax) return mp_fail_noctx(MP_EINVAL, "mp_pn_forward: invalid argument");
    int rc = forward(net, scans, B, false);
    if (rc) return rc;
    PN_CUDA(cudaMemcpyAsync(out, net->o, sizeof(float) * (size_t)B * NOUT, cudaMemcpyDefault, net->stream));
    return MP_OK;
}

int mp_pn_loss_grad(mp_pn* net, const float* scans, const float* targets, int B, float* loss_dev, float* grad_out) {
    if (!net || !scans || !targets || !loss_dev || B < 1 || B > net->Bmax) return mp_fail_noctx(MP_EINVAL, "mp_pn_loss_grad: invalid argument");
    int rc = forward(net, scans, B, true);
    if (rc) return rc;
    cudaStream_t s = net->stream;
    const int64_t rows = (int64_t)B * net->P;
    const float* W = net->param;
    float* G = net->grad;
    PN_CUDA(cudaMemsetAsync(G, 0, sizeof(float) * NPARAM, s));
    PN_CUDA(cudaMemsetAsync(loss_dev, 0, sizeof(float), s));
    k_mdn_loss<<<grid_for(B, 64), 64, 0, s>>>(net->o, targets, B, net->dO, loss_dev);
    // head
    gemm<true, false, EPI_ATOMIC>(s, net->h4, net->dO, G + OW5, nullptr, C4, NOUT, B, C4, NOUT, NOUT);
    colsum(s, net->dO, B, NOUT, G + OB5);
    gemm<false, true, 0>(s, net->dO, W + OW5, net->dh4, nullptr, B, C4, NOUT, NOUT, NOUT, C4);
    k_relu_back<<<grid_for((int64_t)B * C4, 256), 256, 0, s>>>(net->dh4, net->h4, (int64_t)B * C4);
    gemm<true, false, EPI_ATOMIC>(s, net->g, net->dh4, G + OW4, nullptr, C3, C4, B, C3, C4, C4);
    colsum(s, net->dh4, B, C4, G + OB4);
    gemm<false, true, 0>(s, net->dh4, W + OW4, net->dg, nullptr, B, C3, C4, C4, C4, C3);
    // max-pool and the shared layers, on the pooled rows (b, channel) only
    const int64_t rows_c = (int64_t)B * C3;
    k_dw3<<<C3, C2, 0, s>>>(net->dg, net->g, net->gi, net->h2, B, net->P, G + OW3, G + OB3);
    k_pool_rows<<<grid_for(rows_c, 256), 256, 0, s>>>(net->dg, net->g, net->gi, net->xs, net->h1, net->h2, W + OW3, B,
                                                      net->P, net->xc, net->h1c, net->h2c, net->dh2c);
    gemm<true, false, EPI_ATOMIC>(s, net->h1c, net->dh2c, G + OW2, nullptr, C1, C2, (int)rows_c, C1, C2, C2,
                                  splits_for(rows_c, C1, C2));
    colsum(s, net->dh2c, rows_c, C2, G + OB2);
    gemm<false, true, 0>(s, net->dh2c, W + OW2, net->dh1c, nullptr, (int)rows_c, C1, C2, C2, C2, C1);
    k_relu_back<<<grid_for(rows_c * C1, 256), 256, 0, s>>>(net->dh1c, net->h1c, rows_c * C1);
    gemm<true, false, EPI_ATOMIC>(s, net->xc, net->dh1c, G + OW1, nullptr, 3, C1, (int)rows_c, 3, C1, C1,
                                  splits_for(rows_c, 3, C1));
    colsum(s, net->dh1c, rows_c, C1, G + OB1);
    PN_CUDA(cudaGetLastError());
    if (grad_out) PN_CUDA(cudaMemcpyAsync(grad_out, G, sizeof(float) * NPARAM, cudaMemcpyDefault, s));
    return MP_OK;
}

int mp_pn_adam_step(mp_pn* net, float lr, float beta1, float beta2, float eps) {
    if (!net) return mp_fail_noctx(MP_EINVAL, "mp_pn_adam_step: invalid argument");
    net->t += 1;
    const float c1 = 1.f / (1.f - powf(beta1, (float)net->t));
    const float c2 = 1.f / (1.f - powf(beta2, (float)net->t));
    k_adam<<<grid_for(NPARAM, 256), 256, 0, net->stream>>>(net->param, net->grad, net->am, net->av, NPARAM, lr, beta1,
                                                           beta2, eps, c1, c2);
    PN_CUDA(cudaGetLastError());
    if (pack_weights(net)) return pn_fail("weight image", cudaGetLastError());
    return MP_OK;
}

int mp_pn_sample(mp_pn* net, const float* mix, int64_t n, uint64_t seed, float* poses_out) {
    if (!net || !mix || n < 0 || (n > 0 && !poses_out)) return mp_fail_noctx(MP_EINVAL, "mp_pn_sample: invalid argument");
    if (n == 0) return MP_OK;
    k_pn_sample<<<grid_for(n, 256), 256, 0, net->stream>>>(mix, n, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)),
                                                          net->scale, net->offset, poses_out);
    PN_CUDA(cudaGetLastError());
    return MP_OK;
}

int mp_pn_set_precision(mp_pn* net, int precision) {
    if (!net || (precision != MP_PREC_FP32 && precision != MP_PREC_BF16))
        return mp_fail_noctx(MP_EINVAL, "mp_pn_set_precision: invalid argument");
    if (precision == MP_PREC_BF16 && net->P % 128 != 0)
        return mp_fail_noctx(MP_EINVAL, "mp_pn_set_precision: the tensor-core layers take scans of a multiple of "
                                        "128 points, not %d", net->P);
    net->prec = precision;
    if (pack_weights(net)) return pn_fail("weight image", cudaGetLastError());
    return MP_OK;
}

int mp_pn_status(mp_pn* net) {
    if (!net) return mp_fail_noctx(MP_EINVAL, "mp_pn_status: invalid argument");
    int32_t e = 0;
    PN_CUDA(cudaMemcpyAsync(&e, net->err, sizeof(e), cudaMemcpyDeviceToHost, net->stream));
    PN_CUDA(cudaStreamSynchronize(net->stream));
    if (e) {
        PN_CUDA(cudaMemsetAsync(net->err, 0, sizeof(int32_t), net->stream));
        return mp_fail_noctx(MP_ETIMEOUT, "mp_pn: a bounded wait of the tensor-core forward pass gave up");
    }
    return MP_OK;
}

}  // extern "C"
