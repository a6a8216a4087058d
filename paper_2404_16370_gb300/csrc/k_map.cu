// Map and scan preprocessing (Sec. III-C):
//  * GICP point Gaussians: each point's normal from its cov_k nearest points
//    within r_cov (decided by the exact FP32 distance sequence, ties to the
//    smaller index); Sigma = I - (1 - eps_cov) n n^T is carried as n.
//  * the nearest neighbour field m^nnf: per voxel, the nearest valid map point
//    to the voxel centre within r_max (-1 if none).
//  * per-step scan Gaussians and the compaction of the valid scan points into
//    the 32-byte records the likelihood kernel streams through shared memory.
#include "mp_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

// Uniform cell grid of side h over a point set (exact candidate filter: every
// point within distance h of a query lies in the 27 cells around it).
struct CellGridDev {
    float og[3], inv_h;
    int dims[3];
    int64_t ncell;
    uint32_t* start = nullptr;   // ncell + 1
    int32_t* items = nullptr;    // points, grouped by cell
};

__device__ __forceinline__ void cell_coords(const CellGridDev& g, float x, float y, float z, int c[3]) {
    float p[3] = {x, y, z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int v = (int)floorf((p[a] - g.og[a]) * g.inv_h);
        c[a] = min(max(v, -1), g.dims[a]);
    }
}

__global__ void k_cell_count(const float4* __restrict__ pts, const uint8_t* __restrict__ valid, int64_t n,
                             CellGridDev g, int32_t* __restrict__ cell_of, uint32_t* __restrict__ count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (valid && !valid[i]) { cell_of[i] = -1; return; }
    float4 p = pts[i];
    int c[3];
    cell_coords(g, p.x, p.y, p.z, c);
    c[0] = min(max(c[0], 0), g.dims[0] - 1);
    c[1] = min(max(c[1], 0), g.dims[1] - 1);
    c[2] = min(max(c[2], 0), g.dims[2] - 1);
    int64_t ci = ((int64_t)c[2] * g.dims[1] + c[1]) * g.dims[0] + c[0];
    cell_of[i] = (int32_t)ci;
    atomicAdd(&count[ci], 1u);
}

__global__ void k_cell_fill(const int32_t* __restrict__ cell_of, int64_t n, const uint32_t* __restrict__ start,
                            uint32_t* __restrict__ fill, int32_t* __restrict__ items) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = cell_of[i];
    if (c < 0) return;
    uint32_t pos = atomicAdd(&fill[c], 1u);
    items[start[c] + pos] = (int32_t)i;
}

// Sorted insertion of (d, j) into the MP_COVK smallest pairs seen so far
// (order: d, then j). A pair that does not precede the current last one
// cannot enter, and is rejected before the insertion chain.
__device__ __forceinline__ void topk_insert(float (&D)[MP_COVK], int (&J)[MP_COVK], float d, int j) {
    if (!(d < D[MP_COVK - 1] || (d == D[MP_COVK - 1] && j < J[MP_COVK - 1]))) return;
#pragma unroll
    for (int s = 0; s < MP_COVK; ++s) {
        bool lt = (d < D[s]) || (d == D[s] && j < J[s]);
        float td = D[s];
        int tj = J[s];
        D[s] = lt ? d : td;
        J[s] = lt ? j : tj;
        d = lt ? td : d;
        j = lt ? tj : j;
    }
}

// Normal of a 3x3 covariance (FP64): smallest eigenvalue by the closed-form
// trigonometric solution of the characteristic cubic (Smith, CACM 1961),
// refined once by the Rayleigh quotient of its eigenvector; the eigenvector
// is the largest cross product of two rows of (C - lambda I). Sign: the
// largest-magnitude component positive (first index on ties).
__device__ void normal_of_cov(const double C[6], float n_out[3]) {
    // C = (xx, xy, xz, yy, yz, zz)
    double a00 = C[0], a01 = C[1], a02 = C[2], a11 = C[3], a12 = C[4], a22 = C[5];
    double p1 = a01 * a01 + a02 * a02 + a12 * a12;
    double q = (a00 + a11 + a22) / 3.0;
    double b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * p1;
    double lam;
    if (p2 <= 0.0) {
        lam = q;
    } else {
        double p = sqrt(p2 / 6.0);
        double ip = 1.0 / p;
        double c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
        double det = c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02);
        double r = fmin(1.0, fmax(-1.0, 0.5 * det));
        double phi = acos(r) / 3.0;
        lam = q + 2.0 * p * cos(phi + 2.0943951023931954923);   // + 2 pi / 3: the smallest root
    }
    double v[3] = {0, 0, 1};
    for (int it = 0; it < 2; ++it) {
        double r0[3] = {a00 - lam, a01, a02}, r1[3] = {a01, a11 - lam, a12}, r2[3] = {a02, a12, a22 - lam};
        double c[3][3];
        c[0][0] = r0[1] * r1[2] - r0[2] * r1[1]; c[0][1] = r0[2] * r1[0] - r0[0] * r1[2]; c[0][2] = r0[0] * r1[1] - r0[1] * r1[0];
        c[1][0] = r0[1] * r2[2] - r0[2] * r2[1]; c[1][1] = r0[2] * r2[0] - r0[0] * r2[2]; c[1][2] = r0[0] * r2[1] - r0[1] * r2[0];
        c[2][0] = r1[1] * r2[2] - r1[2] * r2[1]; c[2][1] = r1[2] * r2[0] - r1[0] * r2[2]; c[2][2] = r1[0] * r2[1] - r1[1] * r2[0];
        double nn[3];
        int best = 0;
        for (int k = 0; k < 3; ++k) nn[k] = c[k][0] * c[k][0] + c[k][1] * c[k][1] + c[k][2] * c[k][2];
        if (nn[1] > nn[best]) best = 1;
        if (nn[2] > nn[best]) best = 2;
        if (!(nn[best] > 0.0)) break;   // (near) repeated smallest eigenvalue: keep v
        double s = 1.0 / sqrt(nn[best]);
        v[0] = c[best][0] * s; v[1] = c[best][1] * s; v[2] = c[best][2] * s;
        // Rayleigh quotient of the current vector refines lambda
        double Av0 = a00 * v[0] + a01 * v[1] + a02 * v[2];
        double Av1 = a01 * v[0] + a11 * v[1] + a12 * v[2];
        double Av2 = a02 * v[0] + a12 * v[1] + a22 * v[2];
        lam = v[0] * Av0 + v[1] * Av1 + v[2] * Av2;
    }
    int big = 0;
    if (fabs(v[1]) > fabs(v[big])) big = 1;
    if (fabs(v[2]) > fabs(v[big])) big = 2;
    double sg = v[big] < 0 ? -1.0 : 1.0;
    n_out[0] = (float)(sg * v[0]);
    n_out[1] = (float)(sg * v[1]);
    n_out[2] = (float)(sg * v[2]);
}

// FP64 sample covariance of the first m neighbours and the resulting normal.
__device__ void neighbourhood_normal(const float4* __restrict__ pts, const int (&J)[MP_COVK], int m, float n_out[3]) {
    double mx = 0, my = 0, mz = 0;
    for (int s = 0; s < m; ++s) {
        float4 p = pts[J[s]];
        mx += p.x; my += p.y; mz += p.z;
    }
    mx /= m; my /= m; mz /= m;
    double C[6] = {0, 0, 0, 0, 0, 0};
    for (int s = 0; s < m; ++s) {
        float4 p = pts[J[s]];
        double dx = p.x - mx, dy = p.y - my, dz = p.z - mz;
        C[0] += dx * dx; C[1] += dx * dy; C[2] += dx * dz;
        C[3] += dy * dy; C[4] += dy * dz; C[5] += dz * dz;
    }
    for (int a = 0; a < 6; ++a) C[a] /= m;
    normal_of_cov(C, n_out);
}

// Map points: neighbourhoods through the cell grid.
__global__ void k_map_normals(const float4* __restrict__ pts, int64_t n, CellGridDev g, float r2, int k, int kmin,
                              float* __restrict__ normals, uint8_t* __restrict__ valid) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 pi = pts[i];
    float D[MP_COVK];
    int J[MP_COVK];
#pragma unroll
    for (int s = 0; s < MP_COVK; ++s) { D[s] = INFINITY; J[s] = 0x7fffffff; }
    int cnt = 0;
    int c[3];
    cell_coords(g, pi.x, pi.y, pi.z, c);
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int x = c[0] + dx, y = c[1] + dy, z = c[2] + dz;
                if (x < 0 || y < 0 || z < 0 || x >= g.dims[0] || y >= g.dims[1] || z >= g.dims[2]) continue;
                int64_t ci = ((int64_t)z * g.dims[1] + y) * g.dims[0] + x;
                for (uint32_t e = g.start[ci]; e < g.start[ci + 1]; ++e) {
                    int j = g.items[e];
                    float4 pj = pts[j];
                    float d2 = dist2_exact(pi.x, pi.y, pi.z, pj.x, pj.y, pj.z);
                    if (d2 <= r2) {
                        cnt++;
                        topk_insert(D, J, d2, j);
                    }
                }
            }
    int m = min(cnt, k);
    if (m < kmin) {
        valid[i] = 0;
        normals[3 * i] = normals[3 * i + 1] = normals[3 * i + 2] = 0.f;
        return;
    }
    float nv[3];
    neighbourhood_normal(pts, J, m, nv);
    normals[3 * i] = nv[0]; normals[3 * i + 1] = nv[1]; normals[3 * i + 2] = nv[2];
    valid[i] = 1;
}

// Scan points: brute force over the whole scan, staged through shared memory
// in tiles. SCAN_PARTS threads share a point, each scanning every
// SCAN_PARTS-th candidate of a tile with its own top-k, so that a scan of a
// few thousand points still keeps every SM busy; the lists and counts are then
// merged in shared memory (the top-k by (d, j) and the count do not depend on
// the order in which candidates are seen), and one thread per point computes
// the normal.
#define SCAN_TILE 1024
#define SCAN_PARTS 8
#define SCAN_CTA 256
#define SCAN_PTS (SCAN_CTA / SCAN_PARTS)

// Arguments of the per-step scan kernels (raw n x 3 points in, normals,
// validity and the compacted broadcast pairs out).
struct ScanArgs {
    const float* raw;
    int n;
    float r2;
    int k, kmin;
    float4* tmp4;
    float* normals;
    uint8_t* valid;
    float4* pair;
    int32_t* nvalid;
};

struct ScanF4Op {
    using Args = ScanArgs;
    static constexpr int THREADS = 256, MINB = 1;
    static __device__ __forceinline__ void run(const ScanArgs& A, unsigned bx, unsigned) {
        int i = (int)bx * THREADS + threadIdx.x;
        if (i < A.n) A.tmp4[i] = make_float4(A.raw[3 * i], A.raw[3 * i + 1], A.raw[3 * i + 2], 0.f);
    }
};

struct ScanNormalsOp {
    using Args = ScanArgs;
    static constexpr int THREADS = SCAN_CTA, MINB = 1;
    static __device__ __forceinline__ void run(const ScanArgs& A, unsigned bx, unsigned);
};

__device__ __forceinline__ void ScanNormalsOp::run(const ScanArgs& args, unsigned bx, unsigned) {
    const float* __restrict__ raw = args.raw;
    const int n = args.n, k = args.k, kmin = args.kmin;
    const float r2 = args.r2;
    const float4* __restrict__ tmp_pts = args.tmp4;
    float* __restrict__ normals = args.normals;
    uint8_t* __restrict__ valid = args.valid;
    __shared__ float sx[SCAN_TILE], sy[SCAN_TILE], sz[SCAN_TILE];
    __shared__ float Ds[SCAN_PTS][SCAN_PARTS][MP_COVK];
    __shared__ int Js[SCAN_PTS][SCAN_PARTS][MP_COVK];
    __shared__ int cs[SCAN_PTS][SCAN_PARTS];
    const int part = threadIdx.x % SCAN_PARTS, pl = threadIdx.x / SCAN_PARTS;
    const int i = (int)bx * SCAN_PTS + pl;
    float px = 0, py = 0, pz = 0;
    if (i < n) { px = raw[3 * i]; py = raw[3 * i + 1]; pz = raw[3 * i + 2]; }
    float D[MP_COVK];
    int J[MP_COVK];
#pragma unroll
    for (int s = 0; s < MP_COVK; ++s) { D[s] = INFINITY; J[s] = 0x7fffffff; }
    int cnt = 0;
    for (int base = 0; base < n; base += SCAN_TILE) {
        __syncthreads();
        for (int t = threadIdx.x; t < SCAN_TILE && base + t < n; t += SCAN_CTA) {
            sx[t] = raw[3 * (base + t)]; sy[t] = raw[3 * (base + t) + 1]; sz[t] = raw[3 * (base + t) + 2];
        }
        __syncthreads();
        const int m = min(SCAN_TILE, n - base);
        if (i < n) {
            for (int t = part; t < m; t += SCAN_PARTS) {
                float d2 = dist2_exact(px, py, pz, sx[t], sy[t], sz[t]);
                if (d2 <= r2) {
                    cnt++;
                    topk_insert(D, J, d2, base + t);
                }
            }
        }
    }
#pragma unroll
    for (int s = 0; s < MP_COVK; ++s) { Ds[pl][part][s] = D[s]; Js[pl][part][s] = J[s]; }
    cs[pl][part] = cnt;
    __syncthreads();
    // one thread per point (a dense warp) merges the parts and takes the normal
    if (threadIdx.x >= SCAN_PTS) return;
    const int q = threadIdx.x, iq = (int)bx * SCAN_PTS + q;
    if (iq >= n) return;
#pragma unroll
    for (int s = 0; s < MP_COVK; ++s) { D[s] = Ds[q][0][s]; J[s] = Js[q][0][s]; }
    cnt = cs[q][0];
    for (int pp = 1; pp < SCAN_PARTS; ++pp) {
        cnt += cs[q][pp];
        for (int s = 0; s < MP_COVK; ++s) {
            const float d = Ds[q][pp][s];
            if (!(d < INFINITY)) break;   // a part's list is sorted: the rest is empty
            topk_insert(D, J, d, Js[q][pp][s]);
        }
    }
    int m = min(cnt, k);
    if (m < kmin) {
        valid[iq] = 0;
        normals[3 * iq] = normals[3 * iq + 1] = normals[3 * iq + 2] = 0.f;
        return;
    }
#ifdef MP_CHECKED
    for (int s = 0; s < m; ++s)
        if (!MP_DCHECK(J[s] >= 0 && J[s] < n, "scan neighbour index", J[s])) m = 0;
    if (m == 0) {
        valid[iq] = 0;
        return;
    }
#endif
    float nv[3];
    neighbourhood_normal(tmp_pts, J, m, nv);
    normals[3 * iq] = nv[0]; normals[3 * iq + 1] = nv[1]; normals[3 * iq + 2] = nv[2];
    valid[iq] = 1;
}

// Order-preserving compaction of the valid scan points into 48-byte records of
// broadcast pairs (every value twice, the operand layout of the packed pipe);
// one CTA per scan.
struct ScanCompactOp {
    using Args = ScanArgs;
    static constexpr int THREADS = 1024, MINB = 1;
    static __device__ __forceinline__ void run(const ScanArgs& A, unsigned, unsigned);
};

__device__ __forceinline__ void ScanCompactOp::run(const ScanArgs& args, unsigned, unsigned) {
    const float* __restrict__ raw = args.raw;
    const float* __restrict__ normals = args.normals;
    const uint8_t* __restrict__ valid = args.valid;
    const int n = args.n;
    float4* __restrict__ pair = args.pair;
    int32_t* __restrict__ nvalid = args.nvalid;
    __shared__ int warp_tot[32];
    __shared__ int base_s;
    if (threadIdx.x == 0) base_s = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int start = 0; start < n; start += blockDim.x) {
        int i = start + threadIdx.x;
        int f = (i < n && valid[i]) ? 1 : 0;
        unsigned bal = __ballot_sync(0xffffffffu, f);
        int in_warp = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[w] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            if (k < w) off += warp_tot[k];
            tot += warp_tot[k];
        }
        int base = base_s;
        if (f) {
            int o = base + off + in_warp;
            if (!MP_DCHECK(o < n, "compacted scan index", o)) o = 0;
            const float mx = raw[3 * i], my = raw[3 * i + 1], mz = raw[3 * i + 2];
            const float nx = normals[3 * i], ny = normals[3 * i + 1], nz = normals[3 * i + 2];
            pair[3 * o] = make_float4(mx, mx, my, my);
            pair[3 * o + 1] = make_float4(mz, mz, nx, nx);
            pair[3 * o + 2] = make_float4(ny, ny, nz, nz);
        }
        __syncthreads();
        if (threadIdx.x == 0) base_s = base + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *nvalid = base_s;
}

__global__ void __launch_bounds__(256) k_scan_to_float4(const ScanArgs A) { ScanF4Op::run(A, blockIdx.x, 0); }
__global__ void __launch_bounds__(SCAN_CTA) k_scan_normals(const ScanArgs A) { ScanNormalsOp::run(A, blockIdx.x, 0); }
__global__ void __launch_bounds__(1024) k_scan_compact(const ScanArgs A) { ScanCompactOp::run(A, 0, 0); }

// NNF: nearest valid map point to each voxel centre within r_max.
__global__ void k_nnf_build(const float4* __restrict__ pts, CellGridDev g, int nx, int ny, int64_t nvox, float ox,
                            float oy, float oz, float res, float r2, int32_t* __restrict__ nnf) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nvox) return;
    int vx = (int)(idx % nx);
    int64_t r = idx / nx;
    int vy = (int)(r % ny);
    int vz = (int)(r / ny);
    float cx = __fadd_rn(ox, __fmul_rn(__fadd_rn((float)vx, 0.5f), res));
    float cy = __fadd_rn(oy, __fmul_rn(__fadd_rn((float)vy, 0.5f), res));
    float cz = __fadd_rn(oz, __fmul_rn(__fadd_rn((float)vz, 0.5f), res));
    int c[3];
    cell_coords(g, cx, cy, cz, c);
    int best = -1;
    float bd = INFINITY;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int x = c[0] + dx, y = c[1] + dy, z = c[2] + dz;
                if (x < 0 || y < 0 || z < 0 || x >= g.dims[0] || y >= g.dims[1] || z >= g.dims[2]) continue;
                int64_t ci = ((int64_t)z * g.dims[1] + y) * g.dims[0] + x;
                for (uint32_t e = g.start[ci]; e < g.start[ci + 1]; ++e) {
                    int j = g.items[e];
                    float4 p = pts[j];
                    float d2 = dist2_exact(cx, cy, cz, p.x, p.y, p.z);
                    if (d2 <= r2 && (d2 < bd || (d2 == bd && j < best))) { bd = d2; best = j; }
                }
            }
    nnf[idx] = best;
}

// Map records in spatial order: record s holds original point perm[s].
__global__ void k_map_records(const float4* __restrict__ pts, const float* __restrict__ normals,
                              const int32_t* __restrict__ perm, int64_t n, float4* __restrict__ rec) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int64_t i = perm[s];
    float4 p = pts[i];
    rec[2 * s] = make_float4(p.x, p.y, p.z, normals[3 * i]);
    rec[2 * s + 1] = make_float4(normals[3 * i + 1], normals[3 * i + 2], 0.f, 0.f);
}

// Dense NNF entries from original to spatial-order map indices.
__global__ void k_nnf_remap(int32_t* __restrict__ nnf, int64_t nvox, const int32_t* __restrict__ inv) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nvox) return;
    int v = nnf[i];
    if (v >= 0) nnf[i] = inv[v];
}

// NNF values in original map indices.
__global__ void k_nnf_query(const int32_t* __restrict__ nnf, const int32_t* __restrict__ perm, int nx, int ny, int nz,
                            const int32_t* __restrict__ vox, int64_t m, int32_t* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    int x = vox[3 * i], y = vox[3 * i + 1], z = vox[3 * i + 2];
    bool in = x >= 0 && y >= 0 && z >= 0 && x < nx && y < ny && z < nz;
    int s = in ? nnf[((int64_t)z * ny + y) * nx + x] : -1;
    out[i] = s < 0 ? -1 : perm[s];
}

// Spatial order of the map points: Morton code of their cell (side 4 voxels,
// or larger so that 1024 cells cover the box), ties by index.
void morton_order(const std::vector<float>& h, int64_t n, const float lo[3], const float hi[3], float cell,
                  std::vector<int32_t>& perm) {
    auto spread = [](uint32_t x) {
        x &= 0x3ffu;
        x = (x | (x << 16)) & 0x030000FFu;
        x = (x | (x << 8)) & 0x0300F00Fu;
        x = (x | (x << 4)) & 0x030C30C3u;
        x = (x | (x << 2)) & 0x09249249u;
        return x;
    };
    float ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    cell = std::max(cell, ext / 1023.0f);
    std::vector<uint64_t> key((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t c[3];
        for (int a = 0; a < 3; ++a) {
            float f = (h[3 * i + a] - lo[a]) / cell;
            c[a] = (uint32_t)std::min(std::max(f, 0.0f), 1023.0f);
        }
        uint32_t code = spread(c[0]) | (spread(c[1]) << 1) | (spread(c[2]) << 2);
        key[(size_t)i] = ((uint64_t)code << 32) | (uint64_t)i;
    }
    std::sort(key.begin(), key.end());
    perm.resize((size_t)n);
    for (int64_t s = 0; s < n; ++s) perm[(size_t)s] = (int32_t)(key[(size_t)s] & 0xffffffffu);
}

__global__ void k_pts_from_xyz(const float* __restrict__ xyz, int64_t n, float4* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], 0.f);
}

// Builds the cell grid of the (valid) points with cell side h over [lo, hi].
int build_cells(mp_ctx* c, const float4* pts, const uint8_t* valid, int64_t n, float h, const float lo[3],
                const float hi[3], CellGridDev& g, int32_t** cell_of_out) {
    g.inv_h = 1.0f / h;
    g.ncell = 1;
    for (int a = 0; a < 3; ++a) {
        g.og[a] = lo[a] - h;
        g.dims[a] = (int)std::floor((hi[a] - g.og[a]) / h) + 2;
        g.ncell *= g.dims[a];
    }
    if (g.ncell > (int64_t)1 << 30) return mp_fail(c, MP_EINVAL, "cell grid too large (%lld cells)", (long long)g.ncell);
    int32_t* cell_of = nullptr;
    uint32_t *count = nullptr, *fill = nullptr;
    MP_CUDA(c, cudaMalloc(&cell_of, sizeof(int32_t) * (size_t)n));
    MP_CUDA(c, cudaMalloc(&count, sizeof(uint32_t) * (size_t)(g.ncell + 1)));
    MP_CUDA(c, cudaMalloc(&fill, sizeof(uint32_t) * (size_t)(g.ncell + 1)));
    MP_CUDA(c, cudaMalloc(&g.start, sizeof(uint32_t) * (size_t)(g.ncell + 1)));
    MP_CUDA(c, cudaMalloc(&g.items, sizeof(int32_t) * (size_t)n));
    MP_CUDA(c, cudaMemsetAsync(count, 0, sizeof(uint32_t) * (size_t)(g.ncell + 1), c->stream));
    MP_CUDA(c, cudaMemsetAsync(fill, 0, sizeof(uint32_t) * (size_t)(g.ncell + 1), c->stream));
    k_cell_count<<<grid_for(n, 256), 256, 0, c->stream>>>(pts, valid, n, g, cell_of, count);
    MP_LAUNCHED(c);
    int rc = mp_launch_exclusive_scan(c, count, g.start, g.ncell + 1);
    if (rc) return rc;
    k_cell_fill<<<grid_for(n, 256), 256, 0, c->stream>>>(cell_of, n, g.start, fill, g.items);
    MP_LAUNCHED(c);
    MP_CUDA(c, cudaStreamSynchronize(c->stream));
    cudaFree(count);
    cudaFree(fill);
    *cell_of_out = cell_of;
    return MP_OK;
}

void free_cells(CellGridDev& g) {
    cudaFree(g.start);
    cudaFree(g.items);
    g.start = nullptr;
    g.items = nullptr;
}

}  // namespace

// Map preprocessing: normals, validity, NNF geometry (host, FP32 sequence),
// NNF grid and records. xyz_dev: n_map x 3 float32 on the device.
int mp_launch_map_prepare(mp_ctx* c, const float* xyz_dev) {
    int64_t n = c->n_map;
    k_pts_from_xyz<<<grid_for(n, 256), 256, 0, c->stream>>>(xyz_dev, n, c->map_pts);
    MP_LAUNCHED(c);
    // bounding box of all points (exact FP32 min/max on the host)
    std::vector<float> h(3 * (size_t)n);
    MP_CUDA(c, cudaMemcpyAsync(h.data(), xyz_dev, sizeof(float) * 3 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    MP_CUDA(c, cudaStreamSynchronize(c->stream));
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            float v = h[3 * i + a];
            if (!std::isfinite(v)) return mp_fail(c, MP_EINVAL, "map point %lld is not finite", (long long)i);
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
        }
    // normals through a cell grid of side r_cov (+0.1 % margin)
    CellGridDev g;
    int32_t* cell_of = nullptr;
    int rc = build_cells(c, c->map_pts, nullptr, n, c->p.r_cov * 1.001f, lo, hi, g, &cell_of);
    if (rc) return rc;
    float r2c = c->p.r_cov * c->p.r_cov;
    k_map_normals<<<grid_for(n, 128), 128, 0, c->stream>>>(c->map_pts, n, g, r2c, c->p.cov_k, c->p.cov_min,
                                                            c->map_normals, c->map_valid);
    MP_LAUNCHED(c);
    MP_CUDA(c, cudaStreamSynchronize(c->stream));
    free_cells(g);
    cudaFree(cell_of);
    // NNF geometry from the valid points, by the FP32 sequence:
    // o = lo - r_max; n = floor(((hi + r_max) - o) * inv_res) + 1; off = -(o * inv_res)
    std::vector<uint8_t> v((size_t)n);
    MP_CUDA(c, cudaMemcpy(v.data(), c->map_valid, (size_t)n, cudaMemcpyDeviceToHost));
    float vlo[3] = {INFINITY, INFINITY, INFINITY}, vhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int64_t nv = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!v[i]) continue;
        nv++;
        for (int a = 0; a < 3; ++a) {
            vlo[a] = fminf(vlo[a], h[3 * i + a]);
            vhi[a] = fmaxf(vhi[a], h[3 * i + a]);
        }
    }
    c->n_map_valid = nv;
    if (nv == 0) return mp_fail(c, MP_EINVAL, "no map point has %d neighbours within r_cov", c->p.cov_min);
    volatile float res = c->p.nnf_res, rmax = c->p.r_max;
    volatile float inv_res = 1.0f / res;
    c->nnf_inv_res = inv_res;
    c->nnf_voxels = 1;
    for (int a = 0; a < 3; ++a) {
        volatile float o = vlo[a] - rmax;
        volatile float t1 = vhi[a] + rmax;
        volatile float t2 = t1 - o;
        volatile float t3 = t2 * inv_res;
        volatile float po = o * inv_res;
        c->nnf_origin[a] = o;
        c->nnf_dims[a] = (int32_t)std::floor((float)t3) + 1;
        c->nnf_off[a] = -po;
        c->nnf_voxels *= c->nnf_dims[a];
        c->map_lo[a] = vlo[a];
        c->map_hi[a] = vhi[a];
    }
    if (c->nnf_voxels >= ((int64_t)1 << 31))
        return mp_fail(c, MP_EINVAL, "NNF grid of %lld voxels exceeds 2^31", (long long)c->nnf_voxels);
    // dense NNF of original indices (temporary)
    int32_t* dense = nullptr;
    MP_CUDA(c, cudaMalloc(&dense, sizeof(int32_t) * (size_t)c->nnf_voxels));
    rc = build_cells(c, c->map_pts, c->map_valid, n, c->p.r_max * 1.001f, vlo, vhi, g, &cell_of);
    if (rc) { cudaFree(dense); return rc; }
    float r2 = c->p.r_max * c->p.r_max;
    k_nnf_build<<<grid_for(c->nnf_voxels, 256), 256, 0, c->stream>>>(
        c->map_pts, g, c->nnf_dims[0], c->nnf_dims[1], c->nnf_voxels, c->nnf_origin[0], c->nnf_origin[1],
        c->nnf_origin[2], c->p.nnf_res, r2, dense);
    MP_LAUNCHED(c);
    // spatial (Morton) order of the map records: the records that nearby
    // voxels point to share cache lines
    std::vector<int32_t> perm, inv((size_t)n);
    morton_order(h, n, lo, hi, 4.0f * c->p.nnf_res, perm);
    for (int64_t s = 0; s < n; ++s) inv[(size_t)perm[(size_t)s]] = (int32_t)s;
    int32_t* inv_dev = nullptr;
    MP_CUDA(c, cudaMalloc(&c->map_perm, sizeof(int32_t) * (size_t)n));
    MP_CUDA(c, cudaMalloc(&inv_dev, sizeof(int32_t) * (size_t)n));
    MP_CUDA(c, cudaMemcpyAsync(c->map_perm, perm.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    MP_CUDA(c, cudaMemcpyAsync(inv_dev, inv.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    k_map_records<<<grid_for(n, 256), 256, 0, c->stream>>>(c->map_pts, c->map_normals, c->map_perm, n, c->map_rec);
    MP_LAUNCHED(c);
    k_nnf_remap<<<grid_for(c->nnf_voxels, 256), 256, 0, c->stream>>>(dense, c->nnf_voxels, inv_dev);
    MP_LAUNCHED(c);
    MP_CUDA(c, cudaStreamSynchronize(c->stream));
    c->nnf = dense;
    free_cells(g);
    cudaFree(cell_of);
    cudaFree(inv_dev);
    return MP_OK;
}

namespace {

ScanArgs scan_args(mp_ctx* c, const float* raw, int n) {
    ScanArgs A;
    A.raw = raw;
    A.n = n;
    A.r2 = c->p.r_cov * c->p.r_cov;
    A.k = c->p.cov_k;
    A.kmin = c->p.cov_min;
    A.tmp4 = c->scan_tmp4;
    A.normals = c->scan_normals;
    A.valid = c->scan_valid;
    A.pair = c->scan_pair;
    A.nvalid = c->scan_nvalid;
    return A;
}

}  // namespace

// Per-step scan Gaussians (brute-force radius kNN in shared-memory tiles) and
// compaction of the valid points.
int mp_launch_scan_prepare(mp_ctx* c) {
    int n = c->n_scan;
    if (n == 0) {
        MP_CUDA(c, cudaMemsetAsync(c->scan_nvalid, 0, sizeof(int32_t), c->stream));
        return MP_OK;
    }
    const ScanArgs A = scan_args(c, c->scan_raw, n);
    k_scan_to_float4<<<grid_for(n, 256), 256, 0, c->stream>>>(A);
    MP_LAUNCHED(c);
    k_scan_normals<<<grid_for(n, SCAN_PTS), SCAN_CTA, 0, c->stream>>>(A);
    MP_LAUNCHED(c);
    k_scan_compact<<<1, 1024, 0, c->stream>>>(A);
    MP_LAUNCHED(c);
    return MP_OK;
}

// Point Gaussians of an arbitrary point array (the scan-Gaussian kernels
// without the compaction): normals and validity of n points raw_dev (n x 3).
int mp_launch_point_gaussians(mp_ctx* c, const float* raw_dev, int n, float4* tmp4, float* normals, uint8_t* valid) {
    if (n == 0) return MP_OK;
    ScanArgs A = scan_args(c, raw_dev, n);
    A.tmp4 = tmp4;
    A.normals = normals;
    A.valid = valid;
    A.pair = nullptr;
    A.nvalid = nullptr;
    k_scan_to_float4<<<grid_for(n, 256), 256, 0, c->stream>>>(A);
    MP_LAUNCHED(c);
    k_scan_normals<<<grid_for(n, SCAN_PTS), SCAN_CTA, 0, c->stream>>>(A);
    MP_LAUNCHED(c);
    return MP_OK;
}

// Grouped scan stage: every instance's scan is read from the batch's device
// scan buffer; the outputs go to each instance's own scan buffers.
int mp_plan_scan(mp_group* G, int, std::vector<GOp>& plan) {
    std::vector<ScanArgs> tab;
    std::vector<int64_t> b256, b64, b1;
    for (int i = 0; i < G->size(); ++i) {
        const int n = G->n_scan[i];
        tab.push_back(scan_args(G->ctx[i], G->scan_dev + G->scan_off[i], n));
        b256.push_back((n + 255) / 256);
        b64.push_back((n + SCAN_PTS - 1) / SCAN_PTS);
        b1.push_back(1);
    }
    const ScanArgs* t = G->upload(tab);
    unsigned nblk = 0;
    const GBlk* m = G->block_map(b256, &nblk);
    plan_kernel<ScanF4Op>(plan, t, m, nblk);
    m = G->block_map(b64, &nblk);
    plan_kernel<ScanNormalsOp>(plan, t, m, nblk);
    m = G->block_map(b1, &nblk);
    plan_kernel<ScanCompactOp>(plan, t, m, nblk);
    return G->err;
}

int mp_launch_nnf_query(mp_ctx* c, const int32_t* vox_dev, int64_t m, int32_t* out_dev) {
    if (m == 0) return MP_OK;
    k_nnf_query<<<grid_for(m, 256), 256, 0, c->stream>>>(c->nnf, c->map_perm, c->nnf_dims[0], c->nnf_dims[1],
                                                         c->nnf_dims[2], vox_dev, m, out_dev);
    MP_LAUNCHED(c);
    return MP_OK;
}
