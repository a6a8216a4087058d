// Neighbour list update (Sec. III-C, "LSH-based iterative neighbor particle
// search"; Eq. 9, 10; Algorithm 1):
//  * k_lsh_keys   zeta = alpha W^K log(T_LSH^-1 T_i) + delta (FP64), key =
//                 XOR_a floor(zeta_a) * P_a (mod 2^32), bucket = key mod N^B.
//  * radix sort   stable LSD sort of (bucket, id): the distribute loop.
//  * k_merge      one warp per particle: candidates = previous list + a window
//                 of its bucket, d_ij = log(T_i^-1 T_j), s_ij = sum W d^2
//                 (Eq. 7, 8 as printed), keep self + the K-1 smallest (s, j):
//                 the gather loop with the iterative refinement of the lists.
// Also the generic exclusive scan used by the sort and the cell grids.
#include "mp_internal.cuh"

#include <vector>

namespace {

// ---------------------------------------------------------------------------
// exclusive scan (uint32), 4096 elements per block
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_scan_block(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                     int64_t n, uint32_t* __restrict__ block_sums) {
    __shared__ uint32_t warp_tot[32];
    int64_t base = (int64_t)blockIdx.x * 4096 + 4 * threadIdx.x;
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (base + k < n) ? in[base + k] : 0u;
    uint32_t s0 = v[0], s1 = s0 + v[1], s2 = s1 + v[2], tot = s2 + v[3];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t x = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        warp_tot[lane] = x;   // inclusive over warps
    }
    __syncthreads();
    uint32_t excl = inc - tot + (w > 0 ? warp_tot[w - 1] : 0u);
    uint32_t r[4] = {excl, excl + s0, excl + s1, excl + s2};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k < n) out[base + k] = r[k];
    if (threadIdx.x == 1023 && block_sums) block_sums[blockIdx.x] = warp_tot[31];
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int64_t n, const uint32_t* __restrict__ offs) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / 4096];
}

int scan_rec(mp_ctx* c, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp) {
    int64_t nb = (n + 4095) / 4096;
    k_scan_block<<<(unsigned)nb, 1024, 0, c->stream>>>(in, out, n, tmp);
    MP_LAUNCHED(c);
    if (nb > 1) {
        int rc = scan_rec(c, tmp, tmp, nb, tmp + nb);
        if (rc) return rc;
        k_scan_add<<<grid_for(n, 256), 256, 0, c->stream>>>(out, n, tmp);
        MP_LAUNCHED(c);
    }
    return MP_OK;
}

size_t scan_tmp_need(int64_t n) {
    size_t need = 0;
    while (n > 1) {
        n = (n + 4095) / 4096;
        need += (size_t)n;
    }
    return need + 1;
}

// ---------------------------------------------------------------------------
// LSH keys (FP64)
// ---------------------------------------------------------------------------
struct LshArgs {
    double scale[6];   // alpha * W^K diagonal
    uint32_t mask;
    const float4* poses;
    int64_t n;
    const StepDev* sd;
    uint32_t* keys;
    uint32_t* buckets;
};

__device__ __forceinline__ void log_se3_d(double qx, double qy, double qz, double qw, const double t[3], double xi[6]) {
    if (qw < 0) { qx = -qx; qy = -qy; qz = -qz; qw = -qw; }
    double s2 = fma(qz, qz, fma(qy, qy, qx * qx));
    double f;
    if (s2 < 1e-20) f = 2.0 / qw * (1.0 - s2 / (3.0 * qw * qw));
    else {
        double s = sqrt(s2);
        f = 2.0 * atan2(s, qw) / s;
    }
    xi[0] = f * qx; xi[1] = f * qy; xi[2] = f * qz;
    double th2 = fma(xi[2], xi[2], fma(xi[1], xi[1], xi[0] * xi[0]));
    double C;
    if (th2 < 1e-4) C = 1.0 / 12.0 + th2 * (1.0 / 720.0 + th2 * (1.0 / 30240.0));
    else {
        double th = sqrt(th2), sh, ch;
        sincos(0.5 * th, &sh, &ch);
        C = (1.0 - 0.5 * th * ch / sh) / th2;
    }
    double wt[3] = {fma(xi[1], t[2], -xi[2] * t[1]), fma(xi[2], t[0], -xi[0] * t[2]), fma(xi[0], t[1], -xi[1] * t[0])};
    double wwt[3] = {fma(xi[1], wt[2], -xi[2] * wt[1]), fma(xi[2], wt[0], -xi[0] * wt[2]),
                     fma(xi[0], wt[1], -xi[1] * wt[0])};
    for (int a = 0; a < 3; ++a) xi[3 + a] = fma(C, wwt[a], fma(-0.5, wt[a], t[a]));
}

// T_LSH^-1 and delta come from the device-side step values (replayable)
struct LshOp {
    using Args = LshArgs;
    static constexpr int THREADS = 256;
    static __device__ __forceinline__ void run(const LshArgs& A, unsigned bx, unsigned);
};

__device__ __forceinline__ void LshOp::run(const LshArgs& A, unsigned bx, unsigned) {
    const float4* __restrict__ poses = A.poses;
    const StepDev* __restrict__ sd = A.sd;
    const int64_t n = A.n;
    int64_t i = (int64_t)bx * THREADS + threadIdx.x;
    if (i >= n) return;
    float4 a = poses[2 * i], b = poses[2 * i + 1];
    double qx = a.x, qy = a.y, qz = a.z, qw = a.w;
    double nrm = rsqrt(fma(qw, qw, fma(qz, qz, fma(qy, qy, qx * qx))));
    qx *= nrm; qy *= nrm; qz *= nrm; qw *= nrm;
    // relative pose T_LSH^-1 T_i = (Lq (x) q_i, R(Lq) t_i + Lt)
    const double lx = sd->lsh_qinv[0], ly = sd->lsh_qinv[1], lz = sd->lsh_qinv[2], lw = sd->lsh_qinv[3];
    double rw = fma(lw, qw, -fma(lx, qx, fma(ly, qy, lz * qz)));
    double rx = fma(lw, qx, fma(lx, qw, fma(ly, qz, -lz * qy)));
    double ry = fma(lw, qy, fma(-lx, qz, fma(ly, qw, lz * qx)));
    double rz = fma(lw, qz, fma(lx, qy, fma(-ly, qx, lz * qw)));
    const double ti[3] = {b.x, b.y, b.z};
    const double* R = sd->lsh_R;   // rotation of the step's inverse LSH quaternion
    double t[3];
    for (int r = 0; r < 3; ++r)
        t[r] = fma(R[3 * r], ti[0], fma(R[3 * r + 1], ti[1], fma(R[3 * r + 2], ti[2], sd->lsh_tinv[r])));
    double xi[6];
    log_se3_d(rx, ry, rz, rw, t, xi);
    const uint32_t P[6] = {73856093u, 19349663u, 83492791u, 2654435761u, 805459861u, 3674653429u};
    uint32_t key = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        double z = fma(A.scale[k], xi[k], sd->lsh_delta[k]);
        int cell = (int)floor(z);
        key ^= (uint32_t)cell * P[k];
    }
    A.keys[i] = key;
    A.buckets[i] = key & A.mask;
}

__global__ void __launch_bounds__(256) k_lsh_keys(const LshArgs A) { LshOp::run(A, blockIdx.x, 0); }

// ---------------------------------------------------------------------------
// stable LSD radix sort of (bucket, id), 8-bit digits, 2048 elements per block
// ---------------------------------------------------------------------------
// One instance's sort: (key, id) pairs ping-pong between keys[0]/ids[0] and
// keys[1]/ids[1] (pass pss reads pair pss & 1); counts are the digit counts of
// every block, digit-major.
struct SortArgs {
    const uint32_t* buckets;
    uint32_t* keys[2];
    int32_t* ids[2];
    int64_t n;
    uint32_t* counts;
    int nblocks;
    int passes;
    int32_t* sorted_ids;
    int32_t* rank;
    int32_t* blo;
    int32_t* bhi;
};

// A load of sort data. CG: the data may have been written by another CTA
// earlier in the same (persistent) launch, so the load goes through L2
// (ld.global.cg); the read-only path is not coherent within a launch.
template <bool CG, typename T>
__device__ __forceinline__ T ld_sort(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// pass pss (the block map's y index): digit counts of block bx
struct RadixHistOp {
    using Args = SortArgs;
    template <bool CG>
    static __device__ __forceinline__ void body(const SortArgs& A, unsigned bx, unsigned pss);
    static __device__ __forceinline__ void run(const SortArgs& A, unsigned bx, unsigned pss) { body<false>(A, bx, pss); }
};

template <bool CG>
__device__ __forceinline__ void RadixHistOp::body(const SortArgs& A, unsigned bx, unsigned pss) {
    const uint32_t* __restrict__ keys = A.keys[pss & 1];
    const int64_t n = A.n;
    const int shift = (int)pss * MP_RADIX_BITS;
    uint32_t* __restrict__ counts = A.counts;
    const int nblocks = A.nblocks;
    __shared__ uint32_t h[MP_RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)bx * MP_SORT_TILE;
#pragma unroll
    for (int it = 0; it < MP_SORT_TILE / 256; ++it) {
        int64_t idx = base + it * 256 + threadIdx.x;
        if (idx < n) atomicAdd(&h[(ld_sort<CG>(keys + idx) >> shift) & (MP_RADIX - 1)], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + bx] = h[threadIdx.x];
}

// pass pss: stable scatter of block bx by its digit offsets
struct RadixScatterOp {
    using Args = SortArgs;
    template <bool CG>
    static __device__ __forceinline__ void body(const SortArgs& A, unsigned bx, unsigned pss);
    static __device__ __forceinline__ void run(const SortArgs& A, unsigned bx, unsigned pss) { body<false>(A, bx, pss); }
};

template <bool CG>
__device__ __forceinline__ void RadixScatterOp::body(const SortArgs& A, unsigned bx, unsigned pss) {
    const uint32_t* __restrict__ kin = A.keys[pss & 1];
    const int32_t* __restrict__ iin = A.ids[pss & 1];
    uint32_t* __restrict__ kout = A.keys[(pss & 1) ^ 1];
    int32_t* __restrict__ iout = A.ids[(pss & 1) ^ 1];
    const int64_t n = A.n;
    const int shift = (int)pss * MP_RADIX_BITS;
    const uint32_t* __restrict__ offs = A.counts;
    const int nblocks = A.nblocks;
    constexpr int ITEMS = MP_SORT_TILE / 256;   // per lane, consecutive 32-element rows
    __shared__ uint32_t wcnt[8][MP_RADIX];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < 8 * MP_RADIX; d += 256) (&wcnt[0][0])[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)bx * MP_SORT_TILE + (int64_t)w * (32 * ITEMS);
    uint32_t key[ITEMS];
    int32_t id[ITEMS];
    uint32_t loc[ITEMS];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        int64_t idx = base + it * 32 + lane;
        bool ok = idx < n;
        key[it] = ok ? ld_sort<CG>(kin + idx) : 0u;
        id[it] = ok ? ld_sort<CG>(iin + idx) : 0;
        uint32_t dg = ok ? ((key[it] >> shift) & (MP_RADIX - 1)) : MP_RADIX;
        unsigned peers = __match_any_sync(0xffffffffu, dg);
        uint32_t before = ok ? wcnt[w][dg] : 0u;
        __syncwarp();
        int leader = __ffs(peers) - 1;
        if (ok && lane == leader) wcnt[w][dg] = before + __popc(peers);
        __syncwarp();
        loc[it] = before + __popc(peers & lt);
    }
    __syncthreads();
    {   // exclusive prefix over warps, per digit
        uint32_t run = 0;
        for (int k = 0; k < 8; ++k) {
            uint32_t t = wcnt[k][threadIdx.x];
            wcnt[k][threadIdx.x] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        int64_t idx = base + it * 32 + lane;
        if (idx < n) {
            uint32_t dg = (key[it] >> shift) & (MP_RADIX - 1);
            int64_t pos = (int64_t)ld_sort<CG>(offs + (int64_t)dg * nblocks + bx) + wcnt[w][dg] + loc[it];
            if (!MP_DCHECK(pos >= 0 && pos < n, "radix scatter position", pos)) continue;
            kout[pos] = key[it];
            iout[pos] = id[it];
        }
    }
}

__global__ void __launch_bounds__(256) k_radix_hist(const SortArgs A, int pss) { RadixHistOp::run(A, blockIdx.x, pss); }
__global__ void __launch_bounds__(256) k_radix_scatter(const SortArgs A, int pss) {
    RadixScatterOp::run(A, blockIdx.x, pss);
}

__global__ void k_iota(int32_t* __restrict__ a, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = (int32_t)i;
}

// (key, id) pairs of the first pass: (bucket_i, i)
struct SortInitOp {
    using Args = SortArgs;
    static constexpr int THREADS = 256;
    template <bool CG>
    static __device__ __forceinline__ void body(const SortArgs& A, unsigned bx) {
        int64_t i = (int64_t)bx * THREADS + threadIdx.x;
        if (i >= A.n) return;
        A.ids[0][i] = (int32_t)i;
        A.keys[0][i] = ld_sort<CG>(A.buckets + i);
    }
};

// sorted ids out of the last pass's pair, sorted buckets into keys[0]
struct SortFinishOp {
    using Args = SortArgs;
    static constexpr int THREADS = 256;
    template <bool CG>
    static __device__ __forceinline__ void body(const SortArgs& A, unsigned bx) {
        int64_t i = (int64_t)bx * THREADS + threadIdx.x;
        if (i >= A.n) return;
        const int src = A.passes & 1;
        A.sorted_ids[i] = ld_sort<CG>(A.ids[src] + i);
        if (src) A.keys[0][i] = ld_sort<CG>(A.keys[1] + i);
    }
};

// Exclusive scan of one instance's digit counts (256 x nblocks), in place, by
// one CTA of NT threads: 4 NT counts per round with a running carry.
template <int NT, bool CG>
__device__ __forceinline__ void count_scan(const SortArgs& A) {
    constexpr int NW = NT / 32;
    __shared__ uint32_t warp_tot[NW];
    __shared__ uint32_t carry_s;
    const int64_t m = (int64_t)MP_RADIX * A.nblocks;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t base0 = 0; base0 < m; base0 += 4 * NT) {
        const int64_t base = base0 + 4 * threadIdx.x;
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (base + k < m) ? ld_sort<CG>(A.counts + base + k) : 0u;
        const uint32_t s0 = v[0], s1 = s0 + v[1], s2 = s1 + v[2], tot = s2 + v[3];
        uint32_t inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) warp_tot[w] = inc;
        __syncthreads();
        if (w == 0) {
            uint32_t x = lane < NW ? warp_tot[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane < NW) warp_tot[lane] = x;
        }
        __syncthreads();
        const uint32_t carry = carry_s;
        const uint32_t excl = carry + inc - tot + (w > 0 ? warp_tot[w - 1] : 0u);
        const uint32_t r[4] = {excl, excl + s0, excl + s1, excl + s2};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (base + k < m) A.counts[base + k] = r[k];
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + warp_tot[NW - 1];
        __syncthreads();
    }
}

// rank of every particle; [lo, hi) of every present bucket
struct SegmentsOp {
    using Args = SortArgs;
    static constexpr int THREADS = 256;
    template <bool CG>
    static __device__ __forceinline__ void body(const SortArgs& A, unsigned bx) {
        const uint32_t* __restrict__ sk = A.keys[0];
        const int64_t n = A.n;
        int64_t p = (int64_t)bx * THREADS + threadIdx.x;
        if (p >= n) return;
        uint32_t b = ld_sort<CG>(sk + p);
        A.rank[ld_sort<CG>(A.sorted_ids + p)] = (int32_t)p;
        if (p == 0 || ld_sort<CG>(sk + p - 1) != b) A.blo[b] = (int32_t)p;
        if (p == n - 1 || ld_sort<CG>(sk + p + 1) != b) A.bhi[b] = (int32_t)(p + 1);
    }
    static __device__ __forceinline__ void run(const SortArgs& A, unsigned bx, unsigned) { body<false>(A, bx); }
};

__global__ void __launch_bounds__(256) k_segments(const SortArgs A) { SegmentsOp::run(A, blockIdx.x, 0); }

// ---------------------------------------------------------------------------
// visiting order of the likelihood
// ---------------------------------------------------------------------------
// Every particle's sums (Eq. 2-4) are computed by one thread from its own pose
// alone, so the order in which particles are assigned to threads changes no
// result. It decides which NNF sectors the CTAs resident at one time touch:
// in LSH order (Eq. 9-10 hashes pose cells to random buckets) those particles
// are spread over the whole map and nearly every lookup misses L2, while in
// the order of their position the resident particles share the part of the
// grid their scans fall on. The key is the Morton code of the particle's cell
// in a grid of cubes of 2^shift NNF voxels (at most 32 cubes along an axis,
// positions outside the NNF grid clamped to its border); a stable radix sort
// of (key, id) pairs that start in LSH order keeps LSH order within a cell.
struct VisitKeyArgs {
    const float4* poses;
    const int32_t* lsh_order;
    int64_t n;
    float inv_res, off[3];
    int dims[3];
    int shift;
    uint32_t* keys;
    int32_t* ids;
};

// the low 5 bits of v moved to every third bit
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    uint32_t r = 0;
#pragma unroll
    for (int b = 0; b < 5; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

struct VisitKeyOp {
    using Args = VisitKeyArgs;
    static constexpr int THREADS = 256;
    template <bool CG>
    static __device__ __forceinline__ void body(const VisitKeyArgs& A, unsigned bx) {
        const int64_t p = (int64_t)bx * THREADS + threadIdx.x;
        if (p >= A.n) return;
        int32_t i = ld_sort<CG>(A.lsh_order + p);
        if (!MP_DCHECK(i >= 0 && i < A.n, "LSH order entry", i)) i = 0;
        const float4 t = A.poses[2 * (int64_t)i + 1];
        const float x[3] = {t.x, t.y, t.z};
        uint32_t key = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // voxel coordinate as a product and a sum (no contraction in this
            // file); NaN and coordinates below the grid go to cell 0, those
            // above it (the conversion saturates) to the last voxel's cell
            const float f = x[a] * A.inv_res + A.off[a];
            const int v = (f >= 0.f) ? min((int)f, A.dims[a] - 1) : 0;
            key |= spread3((uint32_t)(v >> A.shift)) << a;
        }
        A.keys[p] = key;
        A.ids[p] = i;
    }
    static __device__ __forceinline__ void run(const VisitKeyArgs& A, unsigned bx, unsigned) { body<false>(A, bx); }
};

__global__ void __launch_bounds__(256) k_visit_keys(const VisitKeyArgs A) { VisitKeyOp::run(A, blockIdx.x, 0); }

// ---------------------------------------------------------------------------
// neighbour merge: one warp per particle, 64 candidate slots (2 per lane)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cand_eval(const float4* __restrict__ poses, int j, const Quat& qic, const float Rit[9],
                                          const float ti[3], const float W[2], float d[6], float& s) {
    float4 a, b;
    ld_nc_2x4(poses + 2 * (int64_t)j, a, b);   // the candidate's pose: one 32-byte load
    Quat qr = qmul(qic, Quat{a.x, a.y, a.z, a.w});
    float dt[3] = {b.x - ti[0], b.y - ti[1], b.z - ti[2]};
    float tr[3];
    rot_apply(Rit, dt, tr);
    se3_log_f(qr, tr, d);
    s = W[0] * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) + W[1] * (d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
}

__device__ __forceinline__ void cswap(uint64_t& x, uint64_t y, bool keep_min) {
    x = keep_min ? (x < y ? x : y) : (x > y ? x : y);
}

struct MergeArgs {
    const float4* poses;
    int64_t n;
    int K, C;
    const int32_t* old_ids;
    const uint32_t* buckets;
    const int32_t* sorted_ids;
    const int32_t* rank;
    const int32_t* blo;
    const int32_t* bhi;
    float wr, wt;
    int32_t* ids;
    float* kk;
    float* dd;
};

struct MergeOp {
    using Args = MergeArgs;
    static constexpr int THREADS = 256, MINB = 1;
    static __device__ __forceinline__ void run(const MergeArgs& A, unsigned bx, unsigned);
};

__device__ __forceinline__ void MergeOp::run(const MergeArgs& args, unsigned bx, unsigned) {
    const float4* __restrict__ poses = args.poses;
    const int64_t n = args.n;
    const int K = args.K, C = args.C;
    const int32_t* __restrict__ old_ids = args.old_ids;
    const uint32_t* __restrict__ buckets = args.buckets;
    const int32_t* __restrict__ sorted_ids = args.sorted_ids;
    const int32_t* __restrict__ rank = args.rank;
    const int32_t* __restrict__ blo = args.blo;
    const int32_t* __restrict__ bhi = args.bhi;
    const float wr = args.wr, wt = args.wt;
    int32_t* __restrict__ ids = args.ids;
    float* __restrict__ kk = args.kk;
    float* __restrict__ dd = args.dd;
    int64_t i = ((int64_t)bx * THREADS + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= n) return;
    Quat qi;
    float ti[3];
    load_pose(poses, i, qi, ti);
    float Ri[9], Rit[9];
    quat_rot(qi, Ri);
    Rit[0] = Ri[0]; Rit[1] = Ri[3]; Rit[2] = Ri[6];
    Rit[3] = Ri[1]; Rit[4] = Ri[4]; Rit[5] = Ri[7];
    Rit[6] = Ri[2]; Rit[7] = Ri[5]; Rit[8] = Ri[8];
    Quat qic{-qi.x, -qi.y, -qi.z, qi.w};
    const float W[2] = {wr, wt};
    // element lane: previous list slot `lane`; element 32 + lane: window member
    int ja = -1, jb = -1;
    if (lane < K) {
        int j = old_ids[i * K + lane];
        if (j >= 0 && j != i && MP_DCHECK(j < n, "previous neighbour id", j)) ja = j;
    }
    {
        uint32_t b = buckets[i];
        int lo = blo[b], hi = bhi[b], r = rank[i];
        // The segment table is the last sort's. Buckets of a later LSH draw
        // that no sort followed (a batch whose sort phase gave up at a grid
        // barrier, or stages run out of order) can name an entry that does
        // not hold i, or one never written: the window is then empty.
        if (!(lo >= 0 && lo <= r && r < hi && hi <= n)) {
            lo = 0;
            hi = 0;
        }
        int s0 = r - C / 2;
        int smax = max(lo, hi - C);
        s0 = min(s0, smax);
        s0 = max(s0, lo);
        int e = min(s0 + C, hi);
        if (lane < e - s0) {
            int j = sorted_ids[s0 + lane];
            if (j != i && MP_DCHECK(j >= 0 && j < n, "bucket member id", j)) jb = j;
        }
    }
    float da[6], db[6], sa = 0.f, sb = 0.f;
#pragma unroll
    for (int a = 0; a < 6; ++a) { da[a] = 0.f; db[a] = 0.f; }
    if (ja >= 0) cand_eval(poses, ja, qic, Rit, ti, W, da, sa);
    if (jb >= 0) cand_eval(poses, jb, qic, Rit, ti, W, db, sb);
    uint64_t xa = ja >= 0 ? ((uint64_t)__float_as_uint(sa) << 32) | ((uint64_t)ja << 6) | (uint64_t)lane : ~0ull;
    uint64_t xb = jb >= 0 ? ((uint64_t)__float_as_uint(sb) << 32) | ((uint64_t)jb << 6) | (uint64_t)(32 + lane) : ~0ull;
    // bitonic sort of 64 keys: element e = lane (xa) and e = 32 + lane (xb)
#pragma unroll
    for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 32) {
                // partner of e = lane is e + 32 in the same lane; k = 64: ascending
                uint64_t lo = xa < xb ? xa : xb, hi = xa < xb ? xb : xa;
                xa = lo;
                xb = hi;
            } else {
                uint64_t pa = __shfl_xor_sync(0xffffffffu, xa, j);
                uint64_t pb = __shfl_xor_sync(0xffffffffu, xb, j);
                bool lower = (lane & j) == 0;
                bool up_a = (lane & k) == 0;            // e = lane
                bool up_b = ((32 + lane) & k) == 0;     // e = 32 + lane
                cswap(xa, pa, lower == up_a);
                cswap(xb, pb, lower == up_b);
            }
        }
    }
    // drop duplicates (same s and j are adjacent), keep the first K-1 unique
    uint64_t prev_a = __shfl_up_sync(0xffffffffu, xa, 1);
    uint64_t last_a = __shfl_sync(0xffffffffu, xa, 31);
    uint64_t prev_b = __shfl_up_sync(0xffffffffu, xb, 1);
    if (lane == 0) prev_b = last_a;
    bool va = xa != ~0ull && (lane == 0 || (prev_a >> 6) != (xa >> 6));
    bool vb = xb != ~0ull && ((prev_b >> 6) != (xb >> 6));
    unsigned bal_a = __ballot_sync(0xffffffffu, va), bal_b = __ballot_sync(0xffffffffu, vb);
    const unsigned lt = (1u << lane) - 1u;
    int qa = __popc(bal_a & lt);
    int qb = __popc(bal_a) + __popc(bal_b & lt);
    int nuniq = __popc(bal_a) + __popc(bal_b);
    // fetch d of each element from the lane that evaluated it
    int src_a = (int)(xa & 63u), src_b = (int)(xb & 63u);
    float oa[6], ob[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        float v0 = __shfl_sync(0xffffffffu, da[c], src_a & 31);
        float v1 = __shfl_sync(0xffffffffu, db[c], src_a & 31);
        oa[c] = (src_a >= 32) ? v1 : v0;
        float w0 = __shfl_sync(0xffffffffu, da[c], src_b & 31);
        float w1 = __shfl_sync(0xffffffffu, db[c], src_b & 31);
        ob[c] = (src_b >= 32) ? w1 : w0;
    }
    int64_t row = i * K;
    if (lane == 0) {
        ids[row] = (int32_t)i;
        kk[row] = 1.f;
#pragma unroll
        for (int c = 0; c < 6; ++c) dd[row * 6 + c] = 0.f;
    }
    if (va && qa < K - 1) {
        int64_t o = row + 1 + qa;
        ids[o] = (int32_t)((xa >> 6) & 0x3FFFFFFu);
        kk[o] = expf(-__uint_as_float((uint32_t)(xa >> 32)));
#pragma unroll
        for (int c = 0; c < 6; ++c) dd[o * 6 + c] = oa[c];
    }
    if (vb && qb < K - 1) {
        int64_t o = row + 1 + qb;
        ids[o] = (int32_t)((xb >> 6) & 0x3FFFFFFu);
        kk[o] = expf(-__uint_as_float((uint32_t)(xb >> 32)));
#pragma unroll
        for (int c = 0; c < 6; ++c) dd[o * 6 + c] = ob[c];
    }
    // padding slots
    int slot = lane + 1;
    if (slot < K && slot - 1 >= nuniq) {
        ids[row + slot] = -1;
        kk[row + slot] = 0.f;
#pragma unroll
        for (int c = 0; c < 6; ++c) dd[(row + slot) * 6 + c] = 0.f;
    }
}

__global__ void __launch_bounds__(256) k_merge(const MergeArgs A) { MergeOp::run(A, blockIdx.x, 0); }

// ---------------------------------------------------------------------------
// the LSH / sort / visiting-order phase of a batch as one persistent kernel
// ---------------------------------------------------------------------------
// A cooperative launch whose CTAs take the blocks of every instance in turn,
// with a bounded grid barrier between the sub-steps: keys and first pairs |
// per radix pass: digit counts | count scan (one CTA per instance) | scatter |
// sorted ids | rank and segments | visiting keys | two radix passes of the
// visiting keys | visiting order. The bodies are those of the grouped kernels;
// what a sub-step reads from an earlier one goes through L2.
struct SortPhase {
    const LshArgs* lsh;
    const SortArgs* sort;
    const VisitKeyArgs* vkey;
    const SortArgs* vsort;
    const GBlk* pblk;         // the 256-particle blocks (inst, bx) of every instance
    const GBlk* sblk;         // the 2048-element sort tiles (inst, bx) of every instance
    int32_t* const* err;      // every instance's error word
    int n_pblk, n_sblk, n_inst, max_passes;
    int starve;               // test knob: the first barrier waits for one CTA more than the grid
    GridBar* bar;
    long long budget;
};

constexpr int SORT_PHASE_THREADS = 256;

__device__ __forceinline__ bool sort_phase_sync(const SortPhase& P, unsigned& expect) {
    const bool ok = grid_sync(P.bar, expect, P.budget);
    expect = gridDim.x;
    if (!ok && threadIdx.x == 0)
        for (int k = 0; k < P.n_inst; ++k) atomicOr(P.err[k], MP_ERR_WAIT);
    return ok;
}

// the radix passes [0, passes) of the sorts in tab (one per instance)
__device__ __forceinline__ bool sort_passes(const SortPhase& P, const SortArgs* tab, int passes, unsigned& expect) {
    for (int pss = 0; pss < passes; ++pss) {
        for (int w = blockIdx.x; w < P.n_sblk; w += gridDim.x) {
            const GBlk g = P.sblk[w];
            if (tab[g.inst].passes > pss) RadixHistOp::body<true>(tab[g.inst], (unsigned)g.bx, (unsigned)pss);
            __syncthreads();
        }
        if (!sort_phase_sync(P, expect)) return false;
        for (int k = blockIdx.x; k < P.n_inst; k += gridDim.x) {
            if (tab[k].passes > pss) count_scan<SORT_PHASE_THREADS, true>(tab[k]);
            __syncthreads();
        }
        if (!sort_phase_sync(P, expect)) return false;
        for (int w = blockIdx.x; w < P.n_sblk; w += gridDim.x) {
            const GBlk g = P.sblk[w];
            if (tab[g.inst].passes > pss) RadixScatterOp::body<true>(tab[g.inst], (unsigned)g.bx, (unsigned)pss);
            __syncthreads();
        }
        if (!sort_phase_sync(P, expect)) return false;
    }
    return true;
}

__global__ void __launch_bounds__(SORT_PHASE_THREADS) k_sort_phase(const __grid_constant__ SortPhase P) {
    unsigned expect = gridDim.x + (P.starve ? 1u : 0u);
    for (int w = blockIdx.x; w < P.n_pblk; w += gridDim.x) {
        const GBlk g = P.pblk[w];
        LshOp::run(P.lsh[g.inst], (unsigned)g.bx, 0);
        SortInitOp::body<true>(P.sort[g.inst], (unsigned)g.bx);   // reads the thread's own bucket
    }
    if (!sort_phase_sync(P, expect)) return;
    if (!sort_passes(P, P.sort, P.max_passes, expect)) return;
    for (int w = blockIdx.x; w < P.n_pblk; w += gridDim.x) {
        const GBlk g = P.pblk[w];
        SortFinishOp::body<true>(P.sort[g.inst], (unsigned)g.bx);
    }
    if (!sort_phase_sync(P, expect)) return;
    for (int w = blockIdx.x; w < P.n_pblk; w += gridDim.x) {
        const GBlk g = P.pblk[w];
        SegmentsOp::body<true>(P.sort[g.inst], (unsigned)g.bx);
    }
    if (!sort_phase_sync(P, expect)) return;
    // the visiting keys overwrite the sort buffers the segments just read
    for (int w = blockIdx.x; w < P.n_pblk; w += gridDim.x) {
        const GBlk g = P.pblk[w];
        VisitKeyOp::body<true>(P.vkey[g.inst], (unsigned)g.bx);
    }
    if (!sort_phase_sync(P, expect)) return;
    if (!sort_passes(P, P.vsort, 2, expect)) return;
    for (int w = blockIdx.x; w < P.n_pblk; w += gridDim.x) {
        const GBlk g = P.pblk[w];
        SortFinishOp::body<true>(P.vsort[g.inst], (unsigned)g.bx);
    }
}

}  // namespace

int mp_launch_exclusive_scan(mp_ctx* c, const uint32_t* in, uint32_t* out, int64_t n) {
    // c->scan_tmp holds the block sums of the scans of the step; larger
    // (initialisation-time) scans get a temporary buffer of their own.
    size_t need = scan_tmp_need(n);
    uint32_t* tmp = c->scan_tmp;
    uint32_t* own = nullptr;
    if (need > c->scan_tmp_cap) {
        MP_CUDA(c, cudaMalloc(&own, need * sizeof(uint32_t)));
        tmp = own;
    }
    int rc = scan_rec(c, in, out, n, tmp);
    if (own) {
        cudaStreamSynchronize(c->stream);
        cudaFree(own);
    }
    return rc;
}

namespace {

LshArgs lsh_args(mp_ctx* c, const StepDev* sd) {
    LshArgs A;
    for (int k = 0; k < 6; ++k) A.scale[k] = (double)c->p.alpha * (double)(k < 3 ? c->p.sigma_r : c->p.sigma_t);
    A.mask = c->p.n_buckets_log2 >= 32 ? 0xffffffffu : ((1u << c->p.n_buckets_log2) - 1u);
    A.poses = c->poses[c->cur];
    A.n = c->n;
    A.sd = sd;
    A.keys = c->keys;
    A.buckets = c->buckets;
    return A;
}

SortArgs sort_args(mp_ctx* c) {
    SortArgs A;
    A.buckets = c->buckets;
    A.keys[0] = c->sort_keys[0];
    A.keys[1] = c->sort_keys[1];
    A.ids[0] = c->sort_ids[0];
    A.ids[1] = c->sort_ids[1];
    A.n = c->n;
    A.counts = c->radix_counts;
    A.nblocks = (int)((c->n + MP_SORT_TILE - 1) / MP_SORT_TILE);
    A.passes = (c->p.n_buckets_log2 + MP_RADIX_BITS - 1) / MP_RADIX_BITS;
    A.sorted_ids = c->sorted_ids;
    A.rank = c->rank;
    A.blo = c->seg;
    A.bhi = c->seg + ((int64_t)1 << c->p.n_buckets_log2);
    return A;
}

// 32 cubes or fewer along the longest NNF axis
int visit_shift(const mp_ctx* c) {
    const int dmax = std::max(c->nnf_dims[0], std::max(c->nnf_dims[1], c->nnf_dims[2]));
    int s = 0;
    while ((dmax - 1) >> s >= 32) ++s;
    return s;
}

VisitKeyArgs visit_key_args(mp_ctx* c) {
    VisitKeyArgs A;
    A.poses = c->poses[c->cur];
    A.lsh_order = c->sorted_ids;
    A.n = c->n;
    A.inv_res = c->nnf_inv_res;
    for (int a = 0; a < 3; ++a) {
        A.off[a] = c->nnf_off[a];
        A.dims[a] = c->nnf_dims[a];
    }
    A.shift = visit_shift(c);
    A.keys = c->sort_keys[0];
    A.ids = c->sort_ids[0];
    return A;
}

// the radix passes over the 15-bit visiting keys; SortFinishOp writes the order
SortArgs visit_sort_args(mp_ctx* c) {
    SortArgs A = sort_args(c);
    A.buckets = nullptr;
    A.passes = 2;
    A.sorted_ids = c->visit;
    A.rank = nullptr;
    A.blo = A.bhi = nullptr;
    return A;
}

MergeArgs merge_args(mp_ctx* c, int cur) {
    MergeArgs A;
    A.poses = c->poses[c->cur];
    A.n = c->n;
    A.K = c->p.K;
    A.C = c->p.C;
    A.old_ids = c->nbr_ids[cur];
    A.buckets = c->buckets;
    A.sorted_ids = c->sorted_ids;
    A.rank = c->rank;
    A.blo = c->seg;
    A.bhi = c->seg + ((int64_t)1 << c->p.n_buckets_log2);
    A.wr = c->p.sigma_r;
    A.wt = c->p.sigma_t;
    A.ids = c->nbr_ids[cur ^ 1];
    A.kk = c->nbr_k;
    A.dd = c->nbr_d;
    return A;
}

}  // namespace

int mp_launch_lsh_keys(mp_ctx* c) {
    k_lsh_keys<<<grid_for(c->n, 256), 256, 0, c->stream>>>(lsh_args(c, c->step_dev));
    MP_LAUNCHED(c);
    return MP_OK;
}

int mp_launch_sort(mp_ctx* c) {
    const SortArgs A = sort_args(c);
    const int64_t n = c->n;
    k_iota<<<grid_for(n, 256), 256, 0, c->stream>>>(c->sort_ids[0], n);
    MP_LAUNCHED(c);
    MP_CUDA(c, cudaMemcpyAsync(c->sort_keys[0], c->buckets, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice,
                               c->stream));
    for (int pss = 0; pss < A.passes; ++pss) {
        k_radix_hist<<<A.nblocks, 256, 0, c->stream>>>(A, pss);
        MP_LAUNCHED(c);
        int rc = mp_launch_exclusive_scan(c, c->radix_counts, c->radix_counts, (int64_t)MP_RADIX * A.nblocks);
        if (rc) return rc;
        k_radix_scatter<<<A.nblocks, 256, 0, c->stream>>>(A, pss);
        MP_LAUNCHED(c);
    }
    const int src = A.passes & 1;
    MP_CUDA(c, cudaMemcpyAsync(c->sorted_ids, c->sort_ids[src], sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice,
                               c->stream));
    if (src != 0) {
        MP_CUDA(c, cudaMemcpyAsync(c->sort_keys[0], c->sort_keys[1], sizeof(uint32_t) * (size_t)n,
                                   cudaMemcpyDeviceToDevice, c->stream));
    }
    // sort_keys[0] now holds the sorted buckets; seg[0..2^nb) / seg[2^nb..) hold bucket lo / hi
    k_segments<<<grid_for(n, 256), 256, 0, c->stream>>>(A);
    MP_LAUNCHED(c);
    // the likelihood's visiting order, with the sort buffers free again
    const SortArgs V = visit_sort_args(c);
    k_visit_keys<<<grid_for(n, 256), 256, 0, c->stream>>>(visit_key_args(c));
    MP_LAUNCHED(c);
    for (int pss = 0; pss < V.passes; ++pss) {
        k_radix_hist<<<V.nblocks, 256, 0, c->stream>>>(V, pss);
        MP_LAUNCHED(c);
        int rc = mp_launch_exclusive_scan(c, c->radix_counts, c->radix_counts, (int64_t)MP_RADIX * V.nblocks);
        if (rc) return rc;
        k_radix_scatter<<<V.nblocks, 256, 0, c->stream>>>(V, pss);
        MP_LAUNCHED(c);
    }
    MP_CUDA(c, cudaMemcpyAsync(c->visit, c->sort_ids[V.passes & 1], sizeof(int32_t) * (size_t)n,
                               cudaMemcpyDeviceToDevice, c->stream));
    return MP_OK;
}

int mp_launch_merge(mp_ctx* c) {
    k_merge<<<grid_for(c->n * 32, 256), 256, 0, c->stream>>>(merge_args(c, c->nbr_cur));
    MP_LAUNCHED(c);
    c->nbr_cur ^= 1;
    return MP_OK;
}

// Grid of k_sort_phase on the current device: one CTA per SM. A cooperative
// launch may not exceed the resident CTAs (several per SM), and the phase's
// sub-steps are short, so fewer CTAs make each grid barrier cheaper (measured:
// 4.54 against 4.56 ms a step for 64 small instances).
static unsigned sort_phase_grid_cap() {
    static int cap[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cap[dev]) {
        int sms = 0, per = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sort_phase, SORT_PHASE_THREADS, 0) != cudaSuccess)
            return 0;
        cap[dev] = per > 0 ? sms : 0;
    }
    return (unsigned)cap[dev];
}

// The batch's LSH keys, sort, segments and visiting order: one cooperative
// persistent launch over the particle blocks and sort tiles of all instances
// (its barrier zeroed first).
int mp_plan_lsh_sort(mp_group* G, int, std::vector<GOp>& plan) {
    std::vector<LshArgs> lt;
    std::vector<SortArgs> st, vs;
    std::vector<VisitKeyArgs> vk;
    std::vector<int32_t*> errs;
    std::vector<int64_t> b256, bsort;
    int max_passes = 0;
    for (int i = 0; i < G->size(); ++i) {
        mp_ctx* c = G->ctx[i];
        lt.push_back(lsh_args(c, G->sd_dev + i));
        st.push_back(sort_args(c));
        vk.push_back(visit_key_args(c));
        vs.push_back(visit_sort_args(c));
        errs.push_back(c->dev_error);
        b256.push_back((c->n + 255) / 256);
        bsort.push_back(st.back().nblocks);
        max_passes = std::max(max_passes, std::max(st.back().passes, vs.back().passes));
    }
    SortPhase P = {};
    P.lsh = G->upload(lt);
    P.sort = G->upload(st);
    P.vkey = G->upload(vk);
    P.vsort = G->upload(vs);
    P.err = G->upload(errs);
    unsigned np = 0, ns = 0;
    P.pblk = G->block_map(b256, &np);
    P.sblk = G->block_map(bsort, &ns);
    P.n_pblk = (int)np;
    P.n_sblk = (int)ns;
    P.n_inst = G->size();
    P.max_passes = max_passes;
    P.starve = G->ctx[0]->starve_bar;
    P.bar = static_cast<GridBar*>(G->scratch(sizeof(GridBar)));
    P.budget = G->ctx[0]->wait_budget > 0 ? G->ctx[0]->wait_budget : MP_WAIT_BUDGET;
    const unsigned cap = sort_phase_grid_cap();
    if (G->err) return G->err;
    if (!cap) return MP_ECUDA;
    plan_memset(plan, P.bar, sizeof(GridBar));
    plan_coop(plan, (const void*)k_sort_phase, std::min(std::max(np, ns), cap), SORT_PHASE_THREADS, P);
    return MP_OK;
}

// Grouped merge: graph p reads list nbr_cur ^ p and writes the other.
int mp_plan_merge(mp_group* G, int p, std::vector<GOp>& plan) {
    std::vector<MergeArgs> tab;
    std::vector<int64_t> blocks;
    for (int i = 0; i < G->size(); ++i) {
        mp_ctx* c = G->ctx[i];
        tab.push_back(merge_args(c, c->nbr_cur ^ p));
        blocks.push_back((c->n * 32 + 255) / 256);
    }
    unsigned nblk = 0;
    const GBlk* map = G->block_map(blocks, &nblk);
    plan_kernel<MergeOp>(plan, G->upload(tab), map, nblk);
    return G->err;
}
