// Shared per-point layers of the learned proposal on the 5th-generation tensor
// cores (tcgen05), fused with the max-pool: for every scan point p of sample b
//   h1 = relu(x W1 + b1)      3 -> 64    CUDA cores (FP32, rounded to BF16)
//   h2 = relu(h1 W2 + b2)    64 -> 128   tcgen05.mma, BF16 x BF16 -> FP32 in TMEM
//   h3 = relu(h2 W3 + b3)   128 -> 256   tcgen05.mma, BF16 x BF16 -> FP32 in TMEM
//   g[b][c] = max_p h3[p][c], gi[b][c] = its first point
// (include/mp_proposal.h defines the network). No per-point activation goes to
// global memory unless the caller asks for h1 and h2 (the backward pass reads
// them).
//
// One persistent CTA per SM (256 threads, two warpgroups; 129 KB of shared
// memory keep it alone on its SM, so its 512 TMEM columns are never waited
// for), taking whole samples so that the max-pool stays in registers. Thread
// (row, half), row = tid mod 128 and half = tid / 128, owns tile row `row` (a
// TMEM lane; warps w and w + 4 read the same lane quarter) and half of the
// CUDA-core work of every layer. A sample's points go through in tiles of 128:
//   * thread (r, h) computes channels [32h, 32h + 32) of h1 of point r and
//     writes them, as BF16, into the tile's A operand (K-major, 128-byte
//     swizzle);
//   * one thread issues 4 MMAs (M = 128 points, N = 128, K = 16 each) into
//     TMEM columns [0, 128) and commits them to an mbarrier;
//   * thread (r, h) reads columns [64h, 64h + 64) of row r back (tcgen05.ld),
//     adds b2, applies the ReLU and writes h2 as BF16 into the B operand of
//     the next product;
//   * the third layer is computed transposed, h3^T = W3^T h2^T (two MMA
//     halves of M = 128 channels, N = 128 points, K = 128), into columns
//     [128, 384): TMEM lane r of half h then holds channel 128h + r for all 128
//     points of the tile, so thread (r, h) takes the max over points in
//     registers, in point order (the first maximum), without any cross-thread
//     reduction.
// The BF16 weights W2^T and W3^T are packed once per parameter update into an
// image of exactly this shared-memory layout (k_pn_pack_bf16) and copied in by
// one bulk copy per CTA.
//
// Operand layout (the tcgen05 "128-byte swizzle, K-major" canonical form): a
// block of 128 rows x 64 BF16 columns is 16 KB; rows are 128 bytes, grouped by
// 8 into 1024-byte atoms (the descriptor's stride), and the 16-byte chunk j of
// row r sits at chunk position j XOR (r mod 8). A K step of 16 columns moves
// the descriptor's start address by 32 bytes inside the block.
#include "mp_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace {

constexpr int TC_THREADS = 256;                   // two warpgroups: row = tid % 128, half = tid / 128
constexpr int TC_ROWS = 128;                      // points per tile
constexpr uint32_t SW_BLOCK = 16384;              // 128 rows x 64 BF16, 128-byte swizzle
constexpr uint32_t OFF_W2 = 0;                    // W2^T: n (128) x k (64)
constexpr uint32_t OFF_W3 = OFF_W2 + SW_BLOCK;    // W3^T: [half c / 128][k block] (128 x 64 each)
constexpr uint32_t OFF_H1 = OFF_W3 + 4 * SW_BLOCK;   // h1 tile: p (128) x k (64)
constexpr uint32_t OFF_H2 = OFF_H1 + SW_BLOCK;       // h2 tile: [k block] p (128) x k (64)
constexpr uint32_t SMEM_USED = OFF_H2 + 2 * SW_BLOCK;
constexpr uint32_t SMEM_ALLOC = SMEM_USED + 1024;    // slack to align the operands to 1024 bytes
constexpr uint32_t W_IMAGE_BYTES = 5 * SW_BLOCK;     // W2^T and W3^T, as in shared memory
constexpr uint32_t TMEM_COLS = 512;                  // L2 accumulator [0,128), L3^T halves [128,256), [256,384)

// instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B BF16, both
// K-major, M = 128, N = 128
constexpr uint32_t IDESC_BF16_128x128 = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

// byte offset of element (r, k) of a 128 x 64 BF16 block in the swizzled layout
__host__ __device__ __forceinline__ uint32_t sw128(uint32_t r, uint32_t k) {
    return (r >> 3) * 1024u + (r & 7u) * 128u + ((((k >> 3) ^ r) & 7u) << 4) + (k & 7u) * 2u;
}

// shared-memory matrix descriptor of a swizzled K-major block at shared address saddr
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu)   // start address / 16
           | ((uint64_t)1u << 16)               // leading byte offset (not used by swizzled K-major)
           | ((uint64_t)(1024u >> 4) << 32)     // stride byte offset: one 8-row atom
           | ((uint64_t)1u << 46)               // descriptor version of this architecture family
           | ((uint64_t)2u << 61);              // 128-byte swizzle
}

__device__ __forceinline__ void tc_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// D (TMEM) = A B^T (+ D when accumulate): A, B from shared-memory descriptors
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on the mbarrier once every MMA this thread issued so far has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 64 consecutive FP32 columns of this thread's TMEM lane: four loads in
// flight, one wait. The wait names the destination registers, so that no use
// of them is scheduled before it.
__device__ __forceinline__ void tc_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}
__device__ __forceinline__ void tc_ld64(uint32_t taddr, float v[64]) {
    uint32_t r0[16], r1[16], r2[16], r3[16];
    tc_ld16_issue(taddr, r0);
    tc_ld16_issue(taddr + 16u, r1);
    tc_ld16_issue(taddr + 32u, r2);
    tc_ld16_issue(taddr + 48u, r3);
    tc_wait_ld16(r0);   // waits for all four; the next three only tie their registers to a wait
    tc_wait_ld16(r1);
    tc_wait_ld16(r2);
    tc_wait_ld16(r3);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        v[i] = __uint_as_float(r0[i]);
        v[16 + i] = __uint_as_float(r1[i]);
        v[32 + i] = __uint_as_float(r2[i]);
        v[48 + i] = __uint_as_float(r3[i]);
    }
}

// eight floats from a 16-byte-aligned shared-memory address (two 16-byte loads)
__device__ __forceinline__ void ld8_shared(const float* p, float v[8]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi, float& rlo, float& rhi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);   // .x = lo (low half), .y = hi
    const float2 f = __bfloat1622float2(h);
    rlo = f.x;
    rhi = f.y;
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

// The BF16 image of W2^T and W3^T in the kernel's shared-memory layout.
__global__ void k_pn_pack_bf16(const float* __restrict__ W2, const float* __restrict__ W3,
                               uint8_t* __restrict__ image) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < 64 * 128) {   // W2[k][n]
        const int k = e >> 7, n = e & 127;
        *reinterpret_cast<__nv_bfloat16*>(image + OFF_W2 + sw128(n, k)) = __float2bfloat16_rn(W2[e]);
    }
    if (e < 128 * 256) {   // W3[k][c]
        const int k = e >> 8, c = e & 255;
        const uint32_t blk = (uint32_t)((c >> 7) * 2 + (k >> 6));
        *reinterpret_cast<__nv_bfloat16*>(image + OFF_W3 + blk * SW_BLOCK + sw128(c & 127, k & 63)) =
            __float2bfloat16_rn(W3[e]);
    }
}

struct MlpArgs {
    const float* xs;        // [B * P][3] scaled points
    int B, P;
    const float* W1;        // [3][64]
    const float* b1;        // [64]
    const float* b2;        // [128]
    const float* b3;        // [256]
    const uint8_t* image;   // W2^T, W3^T (BF16, shared-memory layout)
    float* g;               // [B][256]
    int* gi;                // [B][256]
    float* h1_out;          // [B * P][64] or null (values as the MMA saw them)
    float* h2_out;          // [B * P][128] or null
    int32_t* err;           // bit MP_ERR_WAIT: a bounded wait gave up
    long long budget;
};

__global__ void __launch_bounds__(TC_THREADS, 1) k_pn_mlp_tc(const MlpArgs A) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(16) float sW1[3 * 64], sb1[64], sb2[128], sb3[256];   // read 4 at a time
    __shared__ __align__(8) uint64_t bar[3];   // weights copy, layer-2 MMAs, layer-3 MMAs
    __shared__ uint32_t tmem_s;
    const int tid = threadIdx.x, warp = tid >> 5;
    // thread (row, half): TMEM lane / tile row `row`; half of the columns or channels of every layer
    const int row_t = tid & (TC_ROWS - 1), half = tid >> 7;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;   // 1024-aligned operand region (shared address)
    uint8_t* const gb = smem_raw + (base - raw);    // and its generic pointer

    for (int e = tid; e < 3 * 64; e += TC_THREADS) sW1[e] = A.W1[e];
    for (int e = tid; e < 64; e += TC_THREADS) sb1[e] = A.b1[e];
    for (int e = tid; e < 128; e += TC_THREADS) sb2[e] = A.b2[e];
    for (int e = tid; e < 256; e += TC_THREADS) sb3[e] = A.b3[e];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        mbar_fence_init();
    }
    if (warp == 0) {
        tc_alloc(&tmem_s, TMEM_COLS);
        tc_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_s;
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;   // this warp's TMEM lane quarter
    if (tid == 0) {
        mbar_expect_tx(&bar[0], W_IMAGE_BYTES);
        bulk_g2s(gb + OFF_W2, A.image, W_IMAGE_BYTES, &bar[0]);
    }
    bool ok = mbar_wait_bounded(&bar[0], 0, A.budget);
    uint32_t phase = 0;
    const int tiles = A.P / TC_ROWS;
    for (int b = blockIdx.x; b < A.B; b += gridDim.x) {
        float m = -INFINITY;   // channel 128 * half + row_t
        int mi = 0;
        // the tile's points; the next tile's are loaded while the layer-3 MMAs run
        const int64_t row0 = (int64_t)b * A.P + row_t;
        float x0 = A.xs[3 * row0], x1 = A.xs[3 * row0 + 1], x2 = A.xs[3 * row0 + 2];
        for (int t = 0; t < tiles; ++t) {
            if (__syncthreads_or(!ok)) { ok = false; break; }
            const int64_t row = (int64_t)b * A.P + (int64_t)t * TC_ROWS + row_t;
            // layer 1 on the CUDA cores: channels [32 half, 32 half + 32) of point row_t as four 16-byte chunks
#pragma unroll
            for (int c8 = 4 * half; c8 < 4 * half + 4; ++c8) {
                uint32_t w[4];
                float r[8];
                float w0[8], w1[8], w2[8], b0[8];
                ld8_shared(sW1 + c8 * 8, w0);
                ld8_shared(sW1 + 64 + c8 * 8, w1);
                ld8_shared(sW1 + 128 + c8 * 8, w2);
                ld8_shared(sb1 + c8 * 8, b0);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int e = 2 * j;
                    const float v0 = fmaxf(fmaf(x2, w2[e], fmaf(x1, w1[e], fmaf(x0, w0[e], b0[e]))), 0.f);
                    const float v1 = fmaxf(fmaf(x2, w2[e + 1], fmaf(x1, w1[e + 1], fmaf(x0, w0[e + 1], b0[e + 1]))), 0.f);
                    w[j] = bf16x2_bits(v0, v1, r[2 * j], r[2 * j + 1]);
                }
                *reinterpret_cast<uint4*>(gb + OFF_H1 + sw128((uint32_t)row_t, (uint32_t)(c8 * 8))) =
                    make_uint4(w[0], w[1], w[2], w[3]);
                if (A.h1_out) {
                    float4* o = reinterpret_cast<float4*>(A.h1_out + row * 64 + c8 * 8);
                    o[0] = make_float4(r[0], r[1], r[2], r[3]);
                    o[1] = make_float4(r[4], r[5], r[6], r[7]);
                }
            }
            fence_proxy_async_smem();   // the h1 operand (generic writes) before the MMAs read it
            tc_fence_before();          // and the previous tile's TMEM reads before its columns are overwritten
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    tc_mma(tmem, sw128_desc(base + OFF_H1 + 32u * j), sw128_desc(base + OFF_W2 + 32u * j),
                           IDESC_BF16_128x128, j > 0);
                tc_commit(&bar[1]);
            }
            ok = mbar_wait_bounded(&bar[1], phase, A.budget);
            if (__syncthreads_or(!ok)) { ok = false; break; }
            tc_fence_after();
            // layer 2 epilogue: columns [64 half, 64 half + 64) of accumulator row row_t -> h2 (BF16) into
            // the next product's B operand
            float v2[64];
            tc_ld64(tmem + lane_off + 64u * (uint32_t)half, v2);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int j = 4 * half + jj;
                const float* v = v2 + 16 * jj;
                uint32_t w[8];
                float r[16], bb[16];
                ld8_shared(sb2 + 16 * j, bb);
                ld8_shared(sb2 + 16 * j + 8, bb + 8);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    w[i] = bf16x2_bits(fmaxf(v[2 * i] + bb[2 * i], 0.f), fmaxf(v[2 * i + 1] + bb[2 * i + 1], 0.f), r[2 * i],
                                       r[2 * i + 1]);
                const uint32_t blk = OFF_H2 + (uint32_t)(j >> 2) * SW_BLOCK;
                const uint32_t k0 = (uint32_t)(j & 3) * 16u;
                *reinterpret_cast<uint4*>(gb + blk + sw128((uint32_t)row_t, k0)) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4*>(gb + blk + sw128((uint32_t)row_t, k0 + 8)) =
                    make_uint4(w[4], w[5], w[6], w[7]);
                if (A.h2_out) {
                    float4* o = reinterpret_cast<float4*>(A.h2_out + row * 128 + 16 * j);
#pragma unroll
                    for (int q = 0; q < 4; ++q) o[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
                }
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const uint32_t kb = (uint32_t)(j >> 2), kk = 32u * (uint32_t)(j & 3);
                        tc_mma(tmem + 128u + 128u * h, sw128_desc(base + OFF_W3 + (2u * h + kb) * SW_BLOCK + kk),
                               sw128_desc(base + OFF_H2 + kb * SW_BLOCK + kk), IDESC_BF16_128x128, j > 0);
                    }
                tc_commit(&bar[2]);
            }
            if (t + 1 < tiles) {
                const int64_t nrow = row + TC_ROWS;
                x0 = A.xs[3 * nrow];
                x1 = A.xs[3 * nrow + 1];
                x2 = A.xs[3 * nrow + 2];
            }
            ok = mbar_wait_bounded(&bar[2], phase, A.budget);
            if (__syncthreads_or(!ok)) { ok = false; break; }
            tc_fence_after();
            // layer 3 epilogue: lane row_t of half `half` = channel 128 half + row_t, columns = the tile's
            // points in order
            {
                const float bias = sb3[128 * half + row_t];
#pragma unroll 1
                for (int q = 0; q < 2; ++q) {
                    float v[64];
                    tc_ld64(tmem + lane_off + 128u + 128u * (uint32_t)half + 64u * (uint32_t)q, v);
                    // the first maximum of each run of 16 points (four independent chains), then of
                    // the runs in point order: a later value replaces an earlier one only if greater
                    float cm[4];
                    int ci[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        cm[c] = -INFINITY;
                        ci[c] = 0;
#pragma unroll
                        for (int i = 16 * c; i < 16 * c + 16; ++i) {
                            const float y = fmaxf(v[i] + bias, 0.f);
                            if (y > cm[c]) {
                                cm[c] = y;
                                ci[c] = i;
                            }
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (cm[c] > m) {
                            m = cm[c];
                            mi = t * TC_ROWS + 64 * q + ci[c];
                        }
                }
            }
            phase ^= 1u;
        }
        if (!ok) break;
        A.g[(int64_t)b * 256 + 128 * half + row_t] = m;
        A.gi[(int64_t)b * 256 + 128 * half + row_t] = mi;
    }
    if (!ok && tid == 0) atomicOr(A.err, MP_ERR_WAIT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, TMEM_COLS);
}

}  // namespace

size_t mp_pn_tc_image_bytes() { return W_IMAGE_BYTES; }

int mp_pn_tc_pack(const float* W2, const float* W3, uint8_t* image, cudaStream_t s) {
    k_pn_pack_bf16<<<grid_for(128 * 256, 256), 256, 0, s>>>(W2, W3, image);
    return cudaGetLastError() == cudaSuccess ? MP_OK : MP_ECUDA;
}

int mp_pn_tc_forward(const float* xs, int B, int P, const float* W1, const float* b1, const float* b2,
                     const float* b3, const uint8_t* image, float* g, int* gi, float* h1_out, float* h2_out,
                     int32_t* err, long long budget, cudaStream_t s) {
    if (B < 1 || P < TC_ROWS || P % TC_ROWS != 0) return MP_EINVAL;
    static int attr_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MP_ECUDA;
    if (!attr_set[dev]) {
        if (cudaFuncSetAttribute(k_pn_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_ALLOC) !=
            cudaSuccess)
            return MP_ECUDA;
        attr_set[dev] = 1;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MP_ECUDA;
    MlpArgs A;
    A.xs = xs;
    A.B = B;
    A.P = P;
    A.W1 = W1;
    A.b1 = b1;
    A.b2 = b2;
    A.b3 = b3;
    A.image = image;
    A.g = g;
    A.gi = gi;
    A.h1_out = h1_out;
    A.h2_out = h2_out;
    A.err = err;
    A.budget = budget;
    k_pn_mlp_tc<<<(unsigned)std::min(B, sms), TC_THREADS, SMEM_ALLOC, s>>>(A);
    return cudaGetLastError() == cudaSuccess ? MP_OK : MP_ECUDA;
}
