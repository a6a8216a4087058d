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
// Layout: two particles per thread on the packed FP32 pipe (f32x2 fma, mul
// and add; each half rounds exactly as the scalar instruction, so the decision
// sequences are unchanged and the per-pair instruction count roughly halves).
// Every per-pair value is a float2 holding particle a in .x and particle b in
// .y. Particles are visited in the order the sort stage leaves for this
// kernel: by the cell of their position (a coarse Morton order), in LSH order
// within a cell. The CTAs resident at one time then hold particles of one part
// of the map, whose scans fall on a part of the NNF grid that stays in L2
// (in LSH order they are spread over the whole map and most lookups miss L2),
// and neighbouring poses share CTAs, so their NNF and record gathers share L1
// lines once the filter has converged. A thread takes slots p and p + 128 of
// that order, so each half of a warp covers 32 consecutive slots. The scan
// streams through shared memory in chunks of 128 points stored as broadcast
// pairs (48 bytes a point), double-
// buffered with 1-D bulk copies (TMA, cp.async.bulk) completing on mbarriers,
// and every thread of a warp reads the same point. The two dependent gathers
// of a point (NNF entry, then map record) are software-pipelined: the NNF
// entries of point k+2 and the records of point k+1 are in flight while point
// k is accumulated. Accumulation in FP32 registers; the 29 sums of each
// particle are written as a structure of arrays in the visiting order.
#include "mp_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace {

constexpr int LK_THREADS = 128;
constexpr int LK_PER_CTA = 2 * LK_THREADS;
constexpr int LK_CHUNK = 128;   // points per stage: 128 x 48 B = 6 KB (smaller stages leave L1 more room
                                // for the gathers: 3% faster with converged particles than 256)
constexpr int LK_MINB = 3;      // CTAs per SM the register budget must allow (163 registers)
constexpr int LKH_MINB = 4;     // the 16-bit forms: their per-pair values take half the registers, so a
                                // fourth CTA (16 warps per SM) fits in 128 registers

struct LkArgs {
    const float4* poses;
    const int32_t* order;
    int64_t n;
    const float4* scan;      // 3 float4 per valid point, every value twice
    const uint4* scan_h;     // 16-bit forms: 2 uint4 per valid point (broadcast pairs)
    const int32_t* nvalid;
    const int32_t* nnf;      // dense voxel grid of spatial-order map indices
    int nx, ny, nz;
    const float4* rec;
    float c_max;
    float* gn;
    int64_t stride;
    int32_t* err;
    unsigned long long* pairs;
    long long budget;   // cycle limit of each barrier wait
    int starve;         // test knob: announce 16 bytes more than copied for chunk 0
    int split;          // CTAs sharing the scan of one particle block (gridDim.y); > 1 adds atomically
    int64_t n_rec;      // map records (checked builds test the NNF entries against it)
    int scan_cap;       // scan capacity in points (checked builds test the valid count against it)
    // constants as pairs (both halves equal)
    float2 inv2, offx2, offy2, offz2, magic2, m1, half2, half_a2, nhalf_a2, two_eps2, two2, quarter_a2;
};

// Sums of one particle over the scan (map frame, see the file comment).
struct LkAcc {
    float Hww[6];    // (00 01 02 11 12 22)
    float Hwv[9];    // row-major
    float Hvv[6];    // (00 01 02 11 12 22)
    float bw[3], bv[3];
    float ll;
    int cnt;
};

// Rotates the map-frame sums of one particle back to the sensor frame
// (blocks M -> R^T M R, b -> R^T b) and stores the 29 outputs at sorted slot p.
__device__ __forceinline__ void lk_store(const LkArgs& A, const float R[9], const LkAcc& S, int64_t p,
                                         bool add = false) {
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
    for (int f = 0; f < MP_GN; ++f) {
        if (add) atomicAdd(A.gn + (int64_t)f * A.stride + p, out[f]);
        else A.gn[(int64_t)f * A.stride + p] = out[f];
    }
}

// ---------------------------------------------------------------------------
// Packed pair arithmetic.

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

struct Lk2Acc {
    float2 Hww[6], Hwv[9], Hvv[6], bw[3], nbv[3];   // nbv = -bv
    float2 lc;    // sum of the inlier costs
    float2 cnt;   // inlier count
};

struct Lk2Look {
    int ma, mb;
    float2 qx, qy, qz;
};

__device__ __forceinline__ Lk2Look lk2_lookup(const LkArgs& A, const float2 R[9], float2 tx, float2 ty, float2 tz,
                                              const float4* Pp) {
    const float4 p0 = Pp[0], p1 = Pp[1];
    const float2 mx = make_float2(p0.x, p0.y), my = make_float2(p0.z, p0.w), mz = make_float2(p1.x, p1.y);
    Lk2Look L;
    // decision sequence: q~ = fma(R_a2, mz, fma(R_a1, my, R_a0 mx)), q = q~ + t
    L.qx = add2(fma2(R[2], mz, fma2(R[1], my, mul2(R[0], mx))), tx);
    L.qy = add2(fma2(R[5], mz, fma2(R[4], my, mul2(R[3], mx))), ty);
    L.qz = add2(fma2(R[8], mz, fma2(R[7], my, mul2(R[6], mx))), tz);
    // voxel = floor(fma(q, 1/res, off)): round-down add of 1.5 * 2^23
    const float2 fx = __fadd2_rd(fma2(L.qx, A.inv2, A.offx2), A.magic2);
    const float2 fy = __fadd2_rd(fma2(L.qy, A.inv2, A.offy2), A.magic2);
    const float2 fz = __fadd2_rd(fma2(L.qz, A.inv2, A.offz2), A.magic2);
    // unsigned arithmetic: an out-of-range voxel wraps to a large value
    const unsigned vxa = __float_as_uint(fx.x) - 0x4B400000u, vxb = __float_as_uint(fx.y) - 0x4B400000u;
    const unsigned vya = __float_as_uint(fy.x) - 0x4B400000u, vyb = __float_as_uint(fy.y) - 0x4B400000u;
    const unsigned vza = __float_as_uint(fz.x) - 0x4B400000u, vzb = __float_as_uint(fz.y) - 0x4B400000u;
    const bool ina = vxa < (unsigned)A.nx && vya < (unsigned)A.ny && vza < (unsigned)A.nz;
    const bool inb = vxb < (unsigned)A.nx && vyb < (unsigned)A.ny && vzb < (unsigned)A.nz;
    L.ma = -1;
    L.mb = -1;
    if (ina) L.ma = __ldg(A.nnf + (((int)vza * A.ny + (int)vya) * A.nx + (int)vxa));
    if (inb) L.mb = __ldg(A.nnf + (((int)vzb * A.ny + (int)vyb) * A.nx + (int)vxb));
    return L;
}

__device__ __forceinline__ Lk2Look lk2_none() {
    Lk2Look L;
    L.ma = L.mb = -1;
    L.qx = L.qy = L.qz = make_float2(0.f, 0.f);
    return L;
}

// One 32-byte map record (a 32-byte-aligned pair of float4, read-only in the
// kernel) in one 256-bit load: (mu.xyz, w.x) and (w.y, w.z); the last two
// words are padding.
__device__ __forceinline__ void ld_record(const float4* p, float4& r0, float2& r1) {
    float pad0, pad1;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r0.x), "=f"(r0.y), "=f"(r0.z), "=f"(r0.w), "=f"(r1.x), "=f"(r1.y), "=f"(pad0), "=f"(pad1)
        : "l"(p));
}

// Map record of index mm: (mu.xyz, w.x) and (w.y, w.z).
__device__ __forceinline__ void lk2_record(const LkArgs& A, int mm, float4& r0, float2& r1) {
    r0 = make_float4(0.f, 0.f, 0.f, 0.f);
    r1 = make_float2(0.f, 0.f);
    if (mm >= 0 && MP_DCHECK(mm < A.n_rec, "NNF entry beyond the map records", mm)) ld_record(A.rec + 2 * mm, r0, r1);
}

__device__ __forceinline__ void lk2_accumulate(const LkArgs& A, Lk2Acc& S, const float2 R[9], float2 tx, float2 ty,
                                               float2 tz, const float4* Pp, const Lk2Look& L, const float4& ra0,
                                               const float2& ra1, const float4& rb0, const float2& rb1) {
    const float4 p1 = Pp[1], p2 = Pp[2];
    const float2 nx = make_float2(p1.z, p1.w), ny = make_float2(p2.x, p2.y), nz = make_float2(p2.z, p2.w);
    // lever arm q~ = q - t and its negative
    const float2 qtx = fma2(A.m1, tx, L.qx), qty = fma2(A.m1, ty, L.qy), qtz = fma2(A.m1, tz, L.qz);
    const float2 nqx = fma2(A.m1, L.qx, tx), nqy = fma2(A.m1, L.qy, ty), nqz = fma2(A.m1, L.qz, tz);
    // residual e = mu^M - q
    const float2 ex = make_float2(ra0.x - L.qx.x, rb0.x - L.qx.y);
    const float2 ey = make_float2(ra0.y - L.qy.x, rb0.y - L.qy.y);
    const float2 ez = make_float2(ra0.z - L.qz.x, rb0.z - L.qz.y);
    // u = R n (scan normal in the map frame), w = map normal
    const float2 ux = fma2(R[2], nz, fma2(R[1], ny, mul2(R[0], nx)));
    const float2 uy = fma2(R[5], nz, fma2(R[4], ny, mul2(R[3], nx)));
    const float2 uz = fma2(R[8], nz, fma2(R[7], ny, mul2(R[6], nx)));
    // sign of u.w as an explicit fma chain (the library is built without
    // implicit contraction, so every instantiation rounds it the same way)
    const float sga = copysignf(1.f, fmaf(uz.x, ra1.y, fmaf(uy.x, ra1.x, ux.x * ra0.w)));
    const float sgb = copysignf(1.f, fmaf(uz.y, rb1.y, fmaf(uy.y, rb1.x, ux.y * rb0.w)));
    const float2 swx = make_float2(sga * ra0.w, sgb * rb0.w);
    const float2 swy = make_float2(sga * ra1.x, sgb * rb1.x);
    const float2 swz = make_float2(sga * ra1.y, sgb * rb1.y);
    const float2 sx = add2(ux, swx), sy = add2(uy, swy), sz = add2(uz, swz);
    const float2 dx = fma2(A.m1, swx, ux), dy = fma2(A.m1, swy, uy), dz = fma2(A.m1, swz, uz);
    // closed-form Omega = I/2 + as s s^T + ad d d^T
    const float2 dd = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    const float2 ls = fma2(A.half_a2, dd, A.two_eps2);
    const float2 ld = fma2(A.nhalf_a2, dd, A.two2);
    const float2 pr = mul2(ls, ld);
    const float2 rr = mul2(A.quarter_a2, make_float2(__fdividef(1.f, pr.x), __fdividef(1.f, pr.y)));
    const float2 as = mul2(ld, rr), ad = mul2(ls, rr);
    const float2 se = fma2(sz, ez, fma2(sy, ey, mul2(sx, ex)));
    const float2 de = fma2(dz, ez, fma2(dy, ey, mul2(dx, ex)));
    const float2 ee = fma2(ez, ez, fma2(ey, ey, mul2(ex, ex)));
    const float2 cost = fma2(A.half2, ee, fma2(mul2(as, se), se, mul2(mul2(ad, de), de)));
    const bool ia = (L.ma >= 0) && (cost.x <= A.c_max);
    const bool ib = (L.mb >= 0) && (cost.y <= A.c_max);
    const float2 inl = make_float2(ia ? 1.f : 0.f, ib ? 1.f : 0.f);
    S.lc = fma2(inl, cost, S.lc);
    S.cnt = add2(S.cnt, inl);
    const float2 h = mul2(A.half2, inl), Pw = mul2(as, inl), Qw = mul2(ad, inl);
    const float2 Psx = mul2(Pw, sx), Psy = mul2(Pw, sy), Psz = mul2(Pw, sz);
    const float2 Qdx = mul2(Qw, dx), Qdy = mul2(Qw, dy), Qdz = mul2(Qw, dz);
    const float2 Oxx = fma2(Psx, sx, fma2(Qdx, dx, h));
    const float2 Oyy = fma2(Psy, sy, fma2(Qdy, dy, h));
    const float2 Ozz = fma2(Psz, sz, fma2(Qdz, dz, h));
    const float2 Oxy = fma2(Psx, sy, mul2(Qdx, dy));
    const float2 Oxz = fma2(Psx, sz, mul2(Qdx, dz));
    const float2 Oyz = fma2(Psy, sz, mul2(Qdy, dz));
    const float2 gx = fma2(Oxz, ez, fma2(Oxy, ey, mul2(Oxx, ex)));
    const float2 gy = fma2(Oyz, ez, fma2(Oyy, ey, mul2(Oxy, ex)));
    const float2 gz = fma2(Ozz, ez, fma2(Oyz, ey, mul2(Oxz, ex)));
    // Pm = [q~]x Omega (nq = -q~ carries the minus signs)
    const float2 P00 = fma2(qty, Oxz, mul2(nqz, Oxy)), P01 = fma2(qty, Oyz, mul2(nqz, Oyy)),
                 P02 = fma2(qty, Ozz, mul2(nqz, Oyz));
    const float2 P10 = fma2(qtz, Oxx, mul2(nqx, Oxz)), P11 = fma2(qtz, Oxy, mul2(nqx, Oyz)),
                 P12 = fma2(qtz, Oxz, mul2(nqx, Ozz));
    const float2 P20 = fma2(qtx, Oxy, mul2(nqy, Oxx)), P21 = fma2(qtx, Oyy, mul2(nqy, Oxy)),
                 P22 = fma2(qtx, Oyz, mul2(nqy, Oxz));
    // H~_ww += Pm [q~]x^T ; H~_wv += Pm ; H~_vv += Omega
    S.Hww[0] = fma2(qty, P02, fma2(nqz, P01, S.Hww[0]));
    S.Hww[1] = fma2(qtz, P00, fma2(nqx, P02, S.Hww[1]));
    S.Hww[2] = fma2(qtx, P01, fma2(nqy, P00, S.Hww[2]));
    S.Hww[3] = fma2(qtz, P10, fma2(nqx, P12, S.Hww[3]));
    S.Hww[4] = fma2(qtx, P11, fma2(nqy, P10, S.Hww[4]));
    S.Hww[5] = fma2(qtx, P21, fma2(nqy, P20, S.Hww[5]));
    S.Hwv[0] = add2(S.Hwv[0], P00); S.Hwv[1] = add2(S.Hwv[1], P01); S.Hwv[2] = add2(S.Hwv[2], P02);
    S.Hwv[3] = add2(S.Hwv[3], P10); S.Hwv[4] = add2(S.Hwv[4], P11); S.Hwv[5] = add2(S.Hwv[5], P12);
    S.Hwv[6] = add2(S.Hwv[6], P20); S.Hwv[7] = add2(S.Hwv[7], P21); S.Hwv[8] = add2(S.Hwv[8], P22);
    S.Hvv[0] = add2(S.Hvv[0], Oxx); S.Hvv[1] = add2(S.Hvv[1], Oxy); S.Hvv[2] = add2(S.Hvv[2], Oxz);
    S.Hvv[3] = add2(S.Hvv[3], Oyy); S.Hvv[4] = add2(S.Hvv[4], Oyz); S.Hvv[5] = add2(S.Hvv[5], Ozz);
    // b~ = [ g x q~ ; -g ]
    S.bw[0] = fma2(gy, qtz, fma2(gz, nqy, S.bw[0]));
    S.bw[1] = fma2(gz, qtx, fma2(gx, nqz, S.bw[1]));
    S.bw[2] = fma2(gx, qty, fma2(gy, nqx, S.bw[2]));
    S.nbv[0] = add2(S.nbv[0], gx); S.nbv[1] = add2(S.nbv[1], gy); S.nbv[2] = add2(S.nbv[2], gz);
}

// One half (particle a: h = 0, b: h = 1) of the packed sums as scalar sums.
__device__ __forceinline__ LkAcc lk2_half(const LkArgs& A, const Lk2Acc& S, int h, int nv) {
    LkAcc o;
#pragma unroll
    for (int k = 0; k < 6; ++k) { o.Hww[k] = h ? S.Hww[k].y : S.Hww[k].x; o.Hvv[k] = h ? S.Hvv[k].y : S.Hvv[k].x; }
#pragma unroll
    for (int k = 0; k < 9; ++k) o.Hwv[k] = h ? S.Hwv[k].y : S.Hwv[k].x;
#pragma unroll
    for (int k = 0; k < 3; ++k) { o.bw[k] = h ? S.bw[k].y : S.bw[k].x; o.bv[k] = -(h ? S.nbv[k].y : S.nbv[k].x); }
    const float lc = h ? S.lc.y : S.lc.x;
    const float cnt = h ? S.cnt.y : S.cnt.x;
    // log p = -(sum of inlier costs) - c_max * (points that are not inliers)
    o.ll = fmaf(-A.c_max, (float)(nv - (int)cnt), -lc);
    o.cnt = (int)cnt;
    return o;
}

// SPLIT: the scan is shared by A.split CTAs per particle block (partial sums
// added atomically; CTA (bx, by) takes chunks by, by + split, ...); without it
// the loop is the plain one.
template <bool SPLIT>
struct LkOp {
    using Args = LkArgs;
    static constexpr int THREADS = LK_THREADS, MINB = LK_MINB;
    static __device__ __forceinline__ void run(const LkArgs& A, unsigned bxi, unsigned byi);
};

template <bool SPLIT>
__device__ __forceinline__ void LkOp<SPLIT>::run(const LkArgs& A, unsigned bxi, unsigned byi) {
    __shared__ __align__(128) float4 buf[2][3 * LK_CHUNK];
    __shared__ __align__(8) uint64_t bar[2];

    // particles a and b of this thread sit LK_THREADS apart in sorted order,
    // so each half of a warp covers 32 consecutive sorted particles
    const int64_t pa = (int64_t)bxi * LK_PER_CTA + threadIdx.x;
    const int64_t pb = pa + LK_THREADS;
    const bool acta = pa < A.n, actb = pb < A.n;
    int64_t ia = acta ? A.order[pa] : 0, ib = actb ? A.order[pb] : 0;
    if (!MP_DCHECK(ia >= 0 && ia < A.n, "particle order entry", ia)) ia = 0;
    if (!MP_DCHECK(ib >= 0 && ib < A.n, "particle order entry", ib)) ib = 0;
    float2 R[9];
    float2 tx, ty, tz;
    {
        Quat qa, qb;
        float ta[3], tb[3], Ra[9], Rb[9];
        load_pose(A.poses, ia, qa, ta);
        load_pose(A.poses, ib, qb, tb);
        quat_rot_exact(qa, Ra);
        quat_rot_exact(qb, Rb);
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = make_float2(Ra[k], Rb[k]);
        tx = make_float2(ta[0], tb[0]);
        ty = make_float2(ta[1], tb[1]);
        tz = make_float2(ta[2], tb[2]);
    }

    int nv = *A.nvalid;
    if (!MP_DCHECK(nv >= 0 && nv <= A.scan_cap, "valid scan points", nv)) nv = 0;
    const int nchunks = (nv + LK_CHUNK - 1) / LK_CHUNK;
    // scan split: this CTA takes chunks blockIdx.y, blockIdx.y + split, ...
    const int split = SPLIT ? A.split : 1, by = SPLIT ? (int)byi : 0;
    const int nmine = SPLIT ? (by < nchunks ? (nchunks - by + split - 1) / split : 0) : nchunks;
    if (bxi == 0 && by == 0 && threadIdx.x == 0)
        atomicAdd(A.pairs, (unsigned long long)A.n * (unsigned long long)nv);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](float4* dst, uint64_t* b, int cc) {
        int m = min(LK_CHUNK, nv - cc * LK_CHUNK);
        if (!MP_DCHECK(cc >= 0 && m > 0 && ((reinterpret_cast<uintptr_t>(A.scan) & 15) == 0), "scan chunk", cc))
            return;
        uint32_t bytes = (uint32_t)m * 48u;
        fence_proxy_async_smem();   // the block's reads of dst (a reused buffer) before the copy's writes
        mbar_expect_tx(b, bytes + ((A.starve && cc == 0) ? 16u : 0u));
        bulk_g2s(dst, A.scan + 3 * (int64_t)cc * LK_CHUNK, bytes, b);
    };
    if (threadIdx.x == 0) {
        if (nmine > 0) issue(buf[0], &bar[0], by);
        if (nmine > 1) issue(buf[1], &bar[1], by + split);
    }

    Lk2Acc S;
    const float2 z2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 6; ++k) { S.Hww[k] = z2; S.Hvv[k] = z2; }
#pragma unroll
    for (int k = 0; k < 9; ++k) S.Hwv[k] = z2;
#pragma unroll
    for (int k = 0; k < 3; ++k) { S.bw[k] = z2; S.nbv[k] = z2; }
    S.lc = z2;
    S.cnt = z2;

    const bool active = acta;   // acta is false only if actb is false too
    bool failed = false;
    int nv_mine = 0;
    int c = 0;
    for (; c < nmine; ++c) {
        const int b = c & 1;
        const uint32_t parity = (uint32_t)((c >> 1) & 1);
        bool got = mbar_wait_bounded(&bar[b], parity, A.budget);
        if (__syncthreads_or(!got)) { failed = true; break; }
        const int m = min(LK_CHUNK, nv - (by + c * split) * LK_CHUNK);
        nv_mine += m;
        if (active) {
            const float4* P = buf[b];
            // software pipeline over the two dependent gathers: every
            // iteration issues the NNF loads of point k+2 and the record loads
            // of point k+1 before the arithmetic of point k. Invariant at the
            // loop head: sc = point k (records loaded), sb = point k+1 (map
            // indices loaded).
            Lk2Look sb = lk2_none(), sc = lk2_lookup(A, R, tx, ty, tz, P);
            float4 ra0, rb0;
            float2 ra1, rb1;
            lk2_record(A, sc.ma, ra0, ra1);
            lk2_record(A, sc.mb, rb0, rb1);
            if (m > 1) sb = lk2_lookup(A, R, tx, ty, tz, P + 3);
            for (int k = 0; k < m; ++k) {
                const Lk2Look nb = (k + 2 < m) ? lk2_lookup(A, R, tx, ty, tz, P + 3 * (k + 2)) : lk2_none();
                float4 na0, nb0;
                float2 na1, nb1;
                lk2_record(A, sb.ma, na0, na1);
                lk2_record(A, sb.mb, nb0, nb1);
                lk2_accumulate(A, S, R, tx, ty, tz, P + 3 * k, sc, ra0, ra1, rb0, rb1);
                sc = sb;
                sb = nb;
                ra0 = na0; ra1 = na1; rb0 = nb0; rb1 = nb1;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && c + 2 < nmine) issue(buf[b], &bar[b], by + (c + 2) * split);
    }
    if (failed) {
        if (threadIdx.x == 0) {
            atomicOr(A.err, MP_ERR_WAIT);
            for (int k = c; k < min(c + 2, nmine); ++k)
                mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1), A.budget);
        }
        return;
    }
    float Rs[9];
    if (acta) {
#pragma unroll
        for (int k = 0; k < 9; ++k) Rs[k] = R[k].x;
        lk_store(A, Rs, lk2_half(A, S, 0, SPLIT ? nv_mine : nv), pa, SPLIT);
    }
    if (actb) {
#pragma unroll
        for (int k = 0; k < 9; ++k) Rs[k] = R[k].y;
        lk_store(A, Rs, lk2_half(A, S, 1, SPLIT ? nv_mine : nv), pb, SPLIT);
    }
}

template <bool SPLIT>
__global__ void __launch_bounds__(LK_THREADS, LK_MINB) k_likelihood(const LkArgs A) {
    LkOp<SPLIT>::run(A, blockIdx.x, blockIdx.y);
}




// ---------------------------------------------------------------------------
// Mixed-precision form (MP_PREC_BF16 / MP_PREC_FP16): the same two particles
// per thread with the per-pair arithmetic in packed 16-bit pairs. R mu, the
// normal rotation R n, the information matrix, the cost, g = Omega e and
// [q~]x Omega run on bf16x2 / half2; the decision path (q = float(R mu) + t,
// the voxel floor, the NNF), the residual mu^M - q and the lever arm q - t
// stay FP32, and the per-pair products enter the FP32 sums after conversion.
// Masking multiplies only finite values (the information-matrix scalars are
// at most a / (8 eps)); the cost of a point without a map point may overflow
// to +inf in half precision and is only compared, never multiplied.

template <typename H2> struct Half2;
template <> struct Half2<__nv_bfloat162> {
    static __device__ __forceinline__ __nv_bfloat162 from(float2 v) { return __float22bfloat162_rn(v); }
    static __device__ __forceinline__ float2 to(__nv_bfloat162 v) { return __bfloat1622float2(v); }
};
template <> struct Half2<__half2> {
    static __device__ __forceinline__ __half2 from(float2 v) { return __float22half2_rn(v); }
    static __device__ __forceinline__ float2 to(__half2 v) { return __half22float2(v); }
};
template <typename H2>
__device__ __forceinline__ H2 h2_bits(uint32_t u) {
    H2 h;
    memcpy(&h, &u, 4);
    return h;
}
template <typename H2>
__device__ __forceinline__ uint32_t h2_word(H2 h) {
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

// the valid scan as 16-bit broadcast pairs: (mx,mx) (my,my) (mz,mz) (nx,nx) | (ny,ny) (nz,nz) 0 0
template <typename H2>
__global__ void k_scan_to_h2(const float4* __restrict__ pair, const int32_t* __restrict__ nvalid, int n,
                             uint4* __restrict__ out) {
    using T = Half2<H2>;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || i >= *nvalid) return;
    const float4 a = pair[3 * i], b = pair[3 * i + 1], c = pair[3 * i + 2];
    out[2 * i] = make_uint4(h2_word(T::from(make_float2(a.x, a.y))), h2_word(T::from(make_float2(a.z, a.w))),
                            h2_word(T::from(make_float2(b.x, b.y))), h2_word(T::from(make_float2(b.z, b.w))));
    out[2 * i + 1] = make_uint4(h2_word(T::from(make_float2(c.x, c.y))), h2_word(T::from(make_float2(c.z, c.w))), 0u, 0u);
}

template <typename H2>
__device__ __forceinline__ Lk2Look lkh_lookup(const LkArgs& A, const H2 R[9], float2 tx, float2 ty, float2 tz,
                                              const uint4* Pp) {
    using T = Half2<H2>;
    const uint4 p0 = Pp[0];
    const H2 mx = h2_bits<H2>(p0.x), my = h2_bits<H2>(p0.y), mz = h2_bits<H2>(p0.z);
    Lk2Look L;
    L.qx = add2(T::to(__hfma2(R[2], mz, __hfma2(R[1], my, __hmul2(R[0], mx)))), tx);
    L.qy = add2(T::to(__hfma2(R[5], mz, __hfma2(R[4], my, __hmul2(R[3], mx)))), ty);
    L.qz = add2(T::to(__hfma2(R[8], mz, __hfma2(R[7], my, __hmul2(R[6], mx)))), tz);
    const float2 fx = __fadd2_rd(fma2(L.qx, A.inv2, A.offx2), A.magic2);
    const float2 fy = __fadd2_rd(fma2(L.qy, A.inv2, A.offy2), A.magic2);
    const float2 fz = __fadd2_rd(fma2(L.qz, A.inv2, A.offz2), A.magic2);
    // unsigned arithmetic: an out-of-range voxel wraps to a large value
    const unsigned vxa = __float_as_uint(fx.x) - 0x4B400000u, vxb = __float_as_uint(fx.y) - 0x4B400000u;
    const unsigned vya = __float_as_uint(fy.x) - 0x4B400000u, vyb = __float_as_uint(fy.y) - 0x4B400000u;
    const unsigned vza = __float_as_uint(fz.x) - 0x4B400000u, vzb = __float_as_uint(fz.y) - 0x4B400000u;
    const bool ina = vxa < (unsigned)A.nx && vya < (unsigned)A.ny && vza < (unsigned)A.nz;
    const bool inb = vxb < (unsigned)A.nx && vyb < (unsigned)A.ny && vzb < (unsigned)A.nz;
    L.ma = -1;
    L.mb = -1;
    if (ina) L.ma = __ldg(A.nnf + (((int)vza * A.ny + (int)vya) * A.nx + (int)vxa));
    if (inb) L.mb = __ldg(A.nnf + (((int)vzb * A.ny + (int)vyb) * A.nx + (int)vxb));
    return L;
}

template <typename H2>
__device__ __forceinline__ void lkh_accumulate(const LkArgs& A, Lk2Acc& S, const H2 R[9], float2 tx, float2 ty,
                                               float2 tz, const uint4* Pp, const Lk2Look& L, const float4& ra0,
                                               const float2& ra1, const float4& rb0, const float2& rb1) {
    using T = Half2<H2>;
    const uint4 p0 = Pp[0], p1 = Pp[1];
    const H2 nx = h2_bits<H2>(p0.w), ny = h2_bits<H2>(p1.x), nz = h2_bits<H2>(p1.y);
    const H2 half = T::from(make_float2(0.5f, 0.5f));
    const H2 half_a = T::from(A.half_a2), nhalf_a = T::from(A.nhalf_a2), two_eps = T::from(A.two_eps2);
    const H2 two = T::from(A.two2), quarter_a = T::from(A.quarter_a2);
    // FP32 lever arm (and its negative) and residual
    const float2 qtx = fma2(A.m1, tx, L.qx), qty = fma2(A.m1, ty, L.qy), qtz = fma2(A.m1, tz, L.qz);
    const float2 nqx = fma2(A.m1, L.qx, tx), nqy = fma2(A.m1, L.qy, ty), nqz = fma2(A.m1, L.qz, tz);
    const H2 ex = T::from(make_float2(ra0.x - L.qx.x, rb0.x - L.qx.y));
    const H2 ey = T::from(make_float2(ra0.y - L.qy.x, rb0.y - L.qy.y));
    const H2 ez = T::from(make_float2(ra0.z - L.qz.x, rb0.z - L.qz.y));
    const H2 hqx = T::from(qtx), hqy = T::from(qty), hqz = T::from(qtz);
    const H2 hnx = __hneg2(hqx), hny = __hneg2(hqy), hnz = __hneg2(hqz);
    // u = R n, w = map normal
    const H2 ux = __hfma2(R[2], nz, __hfma2(R[1], ny, __hmul2(R[0], nx)));
    const H2 uy = __hfma2(R[5], nz, __hfma2(R[4], ny, __hmul2(R[3], nx)));
    const H2 uz = __hfma2(R[8], nz, __hfma2(R[7], ny, __hmul2(R[6], nx)));
    const H2 wx = T::from(make_float2(ra0.w, rb0.w)), wy = T::from(make_float2(ra1.x, rb1.x));
    const H2 wz = T::from(make_float2(ra1.y, rb1.y));
    const float2 uw = T::to(__hfma2(uz, wz, __hfma2(uy, wy, __hmul2(ux, wx))));
    const H2 sg = T::from(make_float2(copysignf(1.f, uw.x), copysignf(1.f, uw.y)));
    const H2 swx = __hmul2(sg, wx), swy = __hmul2(sg, wy), swz = __hmul2(sg, wz);
    const H2 sx = __hadd2(ux, swx), sy = __hadd2(uy, swy), sz = __hadd2(uz, swz);
    const H2 dx = __hsub2(ux, swx), dy = __hsub2(uy, swy), dz = __hsub2(uz, swz);
    const H2 dd = __hfma2(dz, dz, __hfma2(dy, dy, __hmul2(dx, dx)));
    const H2 ls = __hfma2(half_a, dd, two_eps);
    const H2 ld = __hfma2(nhalf_a, dd, two);
    const H2 rr = __hmul2(quarter_a, h2rcp(__hmul2(ls, ld)));
    const H2 as = __hmul2(ld, rr), ad = __hmul2(ls, rr);
    const H2 se = __hfma2(sz, ez, __hfma2(sy, ey, __hmul2(sx, ex)));
    const H2 de = __hfma2(dz, ez, __hfma2(dy, ey, __hmul2(dx, ex)));
    const H2 ee = __hfma2(ez, ez, __hfma2(ey, ey, __hmul2(ex, ex)));
    const float2 cost = T::to(__hfma2(half, ee, __hfma2(__hmul2(as, se), se, __hmul2(__hmul2(ad, de), de))));
    const bool ia = (L.ma >= 0) && (cost.x <= A.c_max);
    const bool ib = (L.mb >= 0) && (cost.y <= A.c_max);
    S.lc.x += ia ? cost.x : 0.f;
    S.lc.y += ib ? cost.y : 0.f;
    S.cnt = add2(S.cnt, make_float2(ia ? 1.f : 0.f, ib ? 1.f : 0.f));
    const H2 inl = T::from(make_float2(ia ? 1.f : 0.f, ib ? 1.f : 0.f));
    const H2 h = __hmul2(half, inl), Pw = __hmul2(as, inl), Qw = __hmul2(ad, inl);
    const H2 Psx = __hmul2(Pw, sx), Psy = __hmul2(Pw, sy), Psz = __hmul2(Pw, sz);
    const H2 Qdx = __hmul2(Qw, dx), Qdy = __hmul2(Qw, dy), Qdz = __hmul2(Qw, dz);
    const H2 Oxx = __hfma2(Psx, sx, __hfma2(Qdx, dx, h));
    const H2 Oyy = __hfma2(Psy, sy, __hfma2(Qdy, dy, h));
    const H2 Ozz = __hfma2(Psz, sz, __hfma2(Qdz, dz, h));
    const H2 Oxy = __hfma2(Psx, sy, __hmul2(Qdx, dy));
    const H2 Oxz = __hfma2(Psx, sz, __hmul2(Qdx, dz));
    const H2 Oyz = __hfma2(Psy, sz, __hmul2(Qdy, dz));
    const float2 gx = T::to(__hfma2(Oxz, ez, __hfma2(Oxy, ey, __hmul2(Oxx, ex))));
    const float2 gy = T::to(__hfma2(Oyz, ez, __hfma2(Oyy, ey, __hmul2(Oxy, ex))));
    const float2 gz = T::to(__hfma2(Ozz, ez, __hfma2(Oyz, ey, __hmul2(Oxz, ex))));
    // Pm = [q~]x Omega
    const float2 P00 = T::to(__hfma2(hqy, Oxz, __hmul2(hnz, Oxy))), P01 = T::to(__hfma2(hqy, Oyz, __hmul2(hnz, Oyy))),
                 P02 = T::to(__hfma2(hqy, Ozz, __hmul2(hnz, Oyz)));
    const float2 P10 = T::to(__hfma2(hqz, Oxx, __hmul2(hnx, Oxz))), P11 = T::to(__hfma2(hqz, Oxy, __hmul2(hnx, Oyz))),
                 P12 = T::to(__hfma2(hqz, Oxz, __hmul2(hnx, Ozz)));
    const float2 P20 = T::to(__hfma2(hqx, Oxy, __hmul2(hny, Oxx))), P21 = T::to(__hfma2(hqx, Oyy, __hmul2(hny, Oxy))),
                 P22 = T::to(__hfma2(hqx, Oyz, __hmul2(hny, Oxz)));
    // FP32 sums
    S.Hww[0] = fma2(qty, P02, fma2(nqz, P01, S.Hww[0]));
    S.Hww[1] = fma2(qtz, P00, fma2(nqx, P02, S.Hww[1]));
    S.Hww[2] = fma2(qtx, P01, fma2(nqy, P00, S.Hww[2]));
    S.Hww[3] = fma2(qtz, P10, fma2(nqx, P12, S.Hww[3]));
    S.Hww[4] = fma2(qtx, P11, fma2(nqy, P10, S.Hww[4]));
    S.Hww[5] = fma2(qtx, P21, fma2(nqy, P20, S.Hww[5]));
    S.Hwv[0] = add2(S.Hwv[0], P00); S.Hwv[1] = add2(S.Hwv[1], P01); S.Hwv[2] = add2(S.Hwv[2], P02);
    S.Hwv[3] = add2(S.Hwv[3], P10); S.Hwv[4] = add2(S.Hwv[4], P11); S.Hwv[5] = add2(S.Hwv[5], P12);
    S.Hwv[6] = add2(S.Hwv[6], P20); S.Hwv[7] = add2(S.Hwv[7], P21); S.Hwv[8] = add2(S.Hwv[8], P22);
    S.Hvv[0] = add2(S.Hvv[0], T::to(Oxx)); S.Hvv[1] = add2(S.Hvv[1], T::to(Oxy)); S.Hvv[2] = add2(S.Hvv[2], T::to(Oxz));
    S.Hvv[3] = add2(S.Hvv[3], T::to(Oyy)); S.Hvv[4] = add2(S.Hvv[4], T::to(Oyz)); S.Hvv[5] = add2(S.Hvv[5], T::to(Ozz));
    S.bw[0] = fma2(gy, qtz, fma2(gz, nqy, S.bw[0]));
    S.bw[1] = fma2(gz, qtx, fma2(gx, nqz, S.bw[1]));
    S.bw[2] = fma2(gx, qty, fma2(gy, nqx, S.bw[2]));
    S.nbv[0] = add2(S.nbv[0], gx); S.nbv[1] = add2(S.nbv[1], gy); S.nbv[2] = add2(S.nbv[2], gz);
}

template <typename H2, int MINB>
__global__ void __launch_bounds__(LK_THREADS, MINB) k_likelihood_h(const LkArgs A) {
    using T = Half2<H2>;
    __shared__ __align__(128) uint4 buf[2][2 * LK_CHUNK];
    __shared__ __align__(8) uint64_t bar[2];

    const int64_t pa = (int64_t)blockIdx.x * LK_PER_CTA + threadIdx.x;
    const int64_t pb = pa + LK_THREADS;
    const bool acta = pa < A.n, actb = pb < A.n;
    int64_t ia = acta ? A.order[pa] : 0, ib = actb ? A.order[pb] : 0;
    if (!MP_DCHECK(ia >= 0 && ia < A.n, "particle order entry", ia)) ia = 0;
    if (!MP_DCHECK(ib >= 0 && ib < A.n, "particle order entry", ib)) ib = 0;
    H2 R[9];
    float2 tx, ty, tz;
    {
        Quat qa, qb;
        float ta[3], tb[3], Ra[9], Rb[9];
        load_pose(A.poses, ia, qa, ta);
        load_pose(A.poses, ib, qb, tb);
        quat_rot_exact(qa, Ra);
        quat_rot_exact(qb, Rb);
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = T::from(make_float2(Ra[k], Rb[k]));
        tx = make_float2(ta[0], tb[0]);
        ty = make_float2(ta[1], tb[1]);
        tz = make_float2(ta[2], tb[2]);
    }

    int nv = *A.nvalid;
    if (!MP_DCHECK(nv >= 0 && nv <= A.scan_cap, "valid scan points", nv)) nv = 0;
    const int nchunks = (nv + LK_CHUNK - 1) / LK_CHUNK;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(A.pairs, (unsigned long long)A.n * (unsigned long long)nv);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](uint4* dst, uint64_t* b, int cc) {
        int m = min(LK_CHUNK, nv - cc * LK_CHUNK);
        if (!MP_DCHECK(cc >= 0 && m > 0 && ((reinterpret_cast<uintptr_t>(A.scan_h) & 15) == 0), "scan chunk", cc))
            return;
        uint32_t bytes = (uint32_t)m * 32u;
        fence_proxy_async_smem();   // the block's reads of dst (a reused buffer) before the copy's writes
        mbar_expect_tx(b, bytes + ((A.starve && cc == 0) ? 16u : 0u));
        bulk_g2s(dst, A.scan_h + 2 * (int64_t)cc * LK_CHUNK, bytes, b);
    };
    if (threadIdx.x == 0) {
        if (nchunks > 0) issue(buf[0], &bar[0], 0);
        if (nchunks > 1) issue(buf[1], &bar[1], 1);
    }

    Lk2Acc S;
    const float2 z2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 6; ++k) { S.Hww[k] = z2; S.Hvv[k] = z2; }
#pragma unroll
    for (int k = 0; k < 9; ++k) S.Hwv[k] = z2;
#pragma unroll
    for (int k = 0; k < 3; ++k) { S.bw[k] = z2; S.nbv[k] = z2; }
    S.lc = z2;
    S.cnt = z2;

    bool failed = false;
    int c = 0;
    for (; c < nchunks; ++c) {
        const int b = c & 1;
        const uint32_t parity = (uint32_t)((c >> 1) & 1);
        bool got = mbar_wait_bounded(&bar[b], parity, A.budget);
        if (__syncthreads_or(!got)) { failed = true; break; }
        const int m = min(LK_CHUNK, nv - c * LK_CHUNK);
        if (acta) {
            const uint4* P = buf[b];
            // the same two-gather software pipeline as the FP32 form
            Lk2Look sb = lk2_none(), sc = lkh_lookup<H2>(A, R, tx, ty, tz, P);
            float4 ra0, rb0;
            float2 ra1, rb1;
            lk2_record(A, sc.ma, ra0, ra1);
            lk2_record(A, sc.mb, rb0, rb1);
            if (m > 1) sb = lkh_lookup<H2>(A, R, tx, ty, tz, P + 2);
            for (int k = 0; k < m; ++k) {
                const Lk2Look nb = (k + 2 < m) ? lkh_lookup<H2>(A, R, tx, ty, tz, P + 2 * (k + 2)) : lk2_none();
                float4 na0, nb0;
                float2 na1, nb1;
                lk2_record(A, sb.ma, na0, na1);
                lk2_record(A, sb.mb, nb0, nb1);
                lkh_accumulate<H2>(A, S, R, tx, ty, tz, P + 2 * k, sc, ra0, ra1, rb0, rb1);
                sc = sb;
                sb = nb;
                ra0 = na0; ra1 = na1; rb0 = nb0; rb1 = nb1;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && c + 2 < nchunks) issue(buf[b], &bar[b], c + 2);
    }
    if (failed) {
        if (threadIdx.x == 0) {
            atomicOr(A.err, MP_ERR_WAIT);
            for (int k = c; k < min(c + 2, nchunks); ++k)
                mbar_wait_bounded(&bar[k & 1], (uint32_t)((k >> 1) & 1), A.budget);
        }
        return;
    }
    // the FP32 rotation of each particle for the sums' frame change
    float Rs[9];
    Quat q;
    float t[3];
    if (acta) {
        load_pose(A.poses, ia, q, t);
        quat_rot_exact(q, Rs);
        lk_store(A, Rs, lk2_half(A, S, 0, nv), pa);
    }
    if (actb) {
        load_pose(A.poses, ib, q, t);
        quat_rot_exact(q, Rs);
        lk_store(A, Rs, lk2_half(A, S, 1, nv), pb);
    }
}

}  // namespace

namespace {

LkArgs lk_args(mp_ctx* c) {
    LkArgs A;
    A.poses = c->poses[c->cur];
    A.order = c->visit;
    A.n = c->n;
    A.scan = c->scan_pair;
    A.nvalid = c->scan_nvalid;
    A.nnf = c->nnf;
    A.nx = c->nnf_dims[0]; A.ny = c->nnf_dims[1]; A.nz = c->nnf_dims[2];
    A.rec = c->map_rec;
    A.c_max = c->p.c_max;
    A.gn = c->gn;
    A.stride = c->cap;
    A.err = c->dev_error;
    A.budget = c->wait_budget > 0 ? c->wait_budget : MP_WAIT_BUDGET;
    A.starve = c->starve_tx;
    A.pairs = c->pairs;
    const float a = 1.f - c->p.eps_cov;
    auto pair = [](float v) { return make_float2(v, v); };
    A.inv2 = pair(c->nnf_inv_res);
    A.offx2 = pair(c->nnf_off[0]); A.offy2 = pair(c->nnf_off[1]); A.offz2 = pair(c->nnf_off[2]);
    A.magic2 = pair(12582912.0f);   // 1.5 * 2^23: round-down add gives floor in the low bits
    A.m1 = pair(-1.f);
    A.half2 = pair(0.5f);
    A.half_a2 = pair(0.5f * a);
    A.nhalf_a2 = pair(-0.5f * a);
    A.two_eps2 = pair(2.f * c->p.eps_cov);
    A.two2 = pair(2.f);
    A.quarter_a2 = pair(0.25f * a);
    A.scan_h = c->scan_h2;
    A.split = c->lk_split > 1 ? c->lk_split : 1;
    A.n_rec = c->n_map;
    A.scan_cap = c->p.max_scan;
    return A;
}

}  // namespace

int mp_launch_likelihood(mp_ctx* c) {
    LkArgs A = lk_args(c);
    A.split = 1;
    const unsigned grid = grid_for(c->n, LK_PER_CTA);
    if (c->precision == MP_PREC_BF16 || c->precision == MP_PREC_FP16) {
        if (c->n_scan > 0) {
            if (c->precision == MP_PREC_BF16)
                k_scan_to_h2<__nv_bfloat162><<<grid_for(c->n_scan, 256), 256, 0, c->stream>>>(
                    c->scan_pair, c->scan_nvalid, c->n_scan, c->scan_h2);
            else
                k_scan_to_h2<__half2><<<grid_for(c->n_scan, 256), 256, 0, c->stream>>>(c->scan_pair, c->scan_nvalid,
                                                                                        c->n_scan, c->scan_h2);
            MP_LAUNCHED(c);
        }
        if (c->precision == MP_PREC_BF16)
            k_likelihood_h<__nv_bfloat162, LKH_MINB><<<grid, LK_THREADS, 0, c->stream>>>(A);
        else
            k_likelihood_h<__half2, LKH_MINB><<<grid, LK_THREADS, 0, c->stream>>>(A);
    } else {
        // the scan split (a tuning knob for small particle counts): partial
        // sums of each CTA are added into a zeroed output
        A.split = c->lk_split > 1 ? c->lk_split : 1;
        if (A.split > 1) {
            MP_CUDA(c, cudaMemsetAsync(c->gn, 0, sizeof(float) * MP_GN * (size_t)c->cap, c->stream));
            k_likelihood<true><<<dim3(grid, A.split), LK_THREADS, 0, c->stream>>>(A);
        } else {
            k_likelihood<false><<<grid, LK_THREADS, 0, c->stream>>>(A);
        }
    }
    MP_LAUNCHED(c);
    return MP_OK;
}

// Grouped likelihood (FP32): one launch for the instances without a scan
// split, one for those with one (their sums zeroed first, block (bx, by) of
// the map = particle block bx, scan part by).
int mp_plan_likelihood(mp_group* G, int, std::vector<GOp>& plan) {
    std::vector<LkArgs> tab;
    std::vector<int64_t> blocks;
    std::vector<int> plain, split, ys;
    for (int i = 0; i < G->size(); ++i) {
        mp_ctx* c = G->ctx[i];
        tab.push_back(lk_args(c));
        blocks.push_back((c->n + LK_PER_CTA - 1) / LK_PER_CTA);
        ys.push_back(tab.back().split);
        if (tab.back().split > 1) {
            split.push_back(i);
            plan_memset(plan, c->gn, sizeof(float) * MP_GN * (size_t)c->cap);
        } else {
            plain.push_back(i);
        }
    }
    const LkArgs* t = G->upload(tab);
    unsigned nblk = 0;
    if (!plain.empty()) {
        const GBlk* m = G->block_map(blocks, &nblk, plain);
        plan_kernel<LkOp<false>>(plan, t, m, nblk);
    }
    if (!split.empty()) {
        const GBlk* m = G->block_map(blocks, &nblk, split, ys);
        plan_kernel<LkOp<true>>(plan, t, m, nblk);
    }
    return G->err;
}
