// Forward pass of the learned-proposal network on the tensor cores.
//
// The network is 3 -> H -> H -> 1 (ReLU hidden layers, logit output) with
// bf16 weights; activations and sums are float32.  The one dense contraction
// is the hidden H x H layer, z2 = W2 h1, which runs here as a tcgen05 MMA:
// a tile of 128 rows (M) against all H output units (N), K = H.  Layer 1 and
// the head are fused around it:
//   producer warps 4-11 (warp: 8 units of a stage, lane: 4 rows): h1 =
//     relu(W1 f + b1) for 64 units at a time, split into two bf16 planes h1 = hi + lo + r with
//     hi = bf16(h1), lo = bf16(h1 - hi), |r| <= 2^-16 |h1|, written as the
//     K-major A operand (128-byte swizzle) of one pipeline stage;
//   thread 128 issues, per stage, the MMAs of both planes against the bf16
//     W2 slab (resident in shared memory for the whole kernel): the bf16 x
//     bf16 products are exact and accumulate in float32 in tensor memory;
//   epilogue warps 0-3 (thread = TMEM lane = row) read the accumulator,
//     logit = b3 + sum_v w3_v relu(z2_v + b2_v).
// Accumulators are double-buffered (2 x H columns, rounded up to a power of
// 2), so the epilogue of tile t overlaps the layer-1 work and MMAs of tile
// t+1.  Rows come either from a feature array F [n][3] or, for the score
// tables of the learned sweep, are generated in the kernel: row q = (s, x, k) of the table gets the features
// (v_k / 8, 2x - 1, -ln(beta_s) / 4), v_k = -vmax + 2 vmax k / (G - 1).
//
// Every wait is bounded (kWaitNs); a wait that gives up sets the CTA's abort
// flag and records kDevTimeout in the status word, and the kernel returns.
#include <algorithm>
#include <cuda_bf16.h>

#include "hobo_internal.h"
#include "tc_common.cuh"

namespace hobo {

constexpr int kMlpM = 128;          // rows per tile (MMA M)
constexpr int kMlpThreads = 384;    // warps 0-3 epilogue, 4-11 layer 1 + MMA issue
constexpr int kMlpProducers = 256;
constexpr int kMlpStages = 2;       // A-operand stages of 2 planes x 16 KB
constexpr int kMlpKC = 64;          // K per stage (one 128-byte swizzle atom of bf16)

struct MlpTcParams {
    const float* w;        // bf16-rounded weights, flat layout of the network
    int H;
    int64_t n;             // rows
    int64_t tiles;         // ceil(n / 128)
    const float* F;        // [n][3] features, or null for score-table rows
    const float* beta;     // score tables: beta of sweep s
    int G;                 // score tables: points per (sweep, bit value)
    float vmax;
    float* out;            // [n] logits
    int* status;
};

static size_t mlp_tc_smem_bytes(int H)
{
    return 1024 + (size_t)H * H * 2 + (size_t)kMlpStages * 32768 + (size_t)H * 16 + (size_t)H * 8 + 256;
    // (operand B, A stages, layer-1 pairs, head pairs, barriers and flags)
}

__host__ __device__ inline uint32_t tmem_cols_for(int H)
{
    uint32_t c = 32;
    while (c < (uint32_t)(2 * H)) c <<= 1;
    return c;
}

// packed float pairs (element 0 in the low word); the f32x2 arithmetic
// rounds each element exactly as its scalar form
__device__ __forceinline__ uint64_t f32x2(float lo, float hi)
{
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}

__device__ __forceinline__ float lo_f32(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi_f32(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

__device__ __forceinline__ uint64_t fma_f32x2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ uint64_t add_f32x2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint64_t sub_f32x2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_elem, float hi_elem)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__global__ void __launch_bounds__(kMlpThreads, 1)
mlp_forward_tc_kernel(const MlpTcParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int H = p.H;
    const int nKC = H / kMlpKC;
    uint8_t* sB = smem;                                           // nKC x [H rows][128 B]
    uint8_t* sA = sB + (size_t)H * H * 2;                         // kMlpStages x 2 planes x 16 KB
    // layer 1 by unit pairs (u, u+1): [W1[.][0] pair, W1[.][1] pair], [W1[.][2] pair, b1 pair]
    float4* sW1 = reinterpret_cast<float4*>(sA + kMlpStages * 32768);
    // head by column pairs: [b2 pair, w3 pair]
    float4* sBW = sW1 + H;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sBW + H / 2);
    uint64_t* afree = bars;                                       // [kMlpStages]
    uint64_t* accfull = bars + kMlpStages;                        // [2]
    uint64_t* accempty = accfull + 2;                             // [2]
    uint64_t* done = accempty + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    volatile int* never_set = abort_flag + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t oW2 = 4LL * H, ob2 = 4LL * H + (int64_t)H * H, ow3 = ob2 + H, ob3 = ow3 + H;
    const uint32_t ncols = tmem_cols_for(H);
    const uint32_t bstride = ncols / 2;      // columns per accumulator buffer (>= H)

    // ---- W2 as the bf16 B operand (n = output unit v, k = input unit u),
    // K-major, 128-byte swizzle; the weights are bf16 values already, so the
    // conversion is exact.
    {
        const int cpr = H / 8;                       // 16-byte chunks per row of W2
        for (int q = threadIdx.x; q < H * cpr; q += kMlpThreads) {
            const int v = q / cpr, cg = q % cpr;
            const int kc = cg >> 3, c = cg & 7;
            const float4* src = reinterpret_cast<const float4*>(p.w + oW2 + (int64_t)v * H + cg * 8);
            const float4 a = __ldg(src), b = __ldg(src + 1);
            uint8_t* dst = sB + (size_t)kc * H * 128 + (v >> 3) * 1024 + (v & 7) * 128 + ((c ^ (v & 7)) << 4);
            *reinterpret_cast<uint4*>(dst) =
                make_uint4(pack_bf16x2(a.x, a.y), pack_bf16x2(a.z, a.w), pack_bf16x2(b.x, b.y), pack_bf16x2(b.z, b.w));
        }
        for (int j = threadIdx.x; j < H / 2; j += kMlpThreads) {
            const int u = 2 * j;
            sW1[2 * j] = make_float4(__ldg(p.w + 3 * u), __ldg(p.w + 3 * u + 3), __ldg(p.w + 3 * u + 1),
                                     __ldg(p.w + 3 * u + 4));
            sW1[2 * j + 1] = make_float4(__ldg(p.w + 3 * u + 2), __ldg(p.w + 3 * u + 5), __ldg(p.w + 3LL * H + u),
                                         __ldg(p.w + 3LL * H + u + 1));
            sBW[j] = make_float4(__ldg(p.w + ob2 + u), __ldg(p.w + ob2 + u + 1), __ldg(p.w + ow3 + u),
                                 __ldg(p.w + ow3 + u + 1));
        }
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMlpStages; ++s) mbar_init(&afree[s], 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(&accfull[s], 1);
            mbar_init(&accempty[s], 4);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *never_set = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_proxy_async_smem();
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    const float b3 = __ldg(p.w + ob3);

    if (warp >= 4) {
        // ---- layer 1 into the A operand.  Producer warp c (0..7) computes
        // units c * 8 .. c * 8 + 7 of every stage, so its weights are the
        // same for all lanes; lane L takes the four rows
        // (L & 7) + 8 * (4 * (L >> 3) + i), i = 0..3, so that the eight
        // lanes storing one row's chunk position hit eight different
        // 16-byte bank groups of the 128-byte swizzle.  MMA issue by thread 128.
        const int c = warp - 4;
        int rr[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) rr[i] = (lane & 7) + 8 * (4 * (lane >> 3) + i);
        const uint32_t idesc = idesc_bf16(kMlpM, H);
        int cc = 0;                                   // stages used so far
        bool fail = false;
        int64_t lt = 0;
        // features of row r of a tile (zeros past the last row)
        auto features = [&](int64_t tile, int r, float& f0, float& f1, float& f2) {
            const int64_t row = tile * kMlpM + r;
            f0 = f1 = f2 = 0.f;
            if (tile >= p.tiles || row >= p.n) return;
            if (p.F) {
                f0 = __ldg(p.F + row * 3);
                f1 = __ldg(p.F + row * 3 + 1);
                f2 = __ldg(p.F + row * 3 + 2);
            } else {
                const int s = (int)(row / (2 * p.G));
                const int x = (int)((row / p.G) % 2);
                const int k = (int)(row % p.G);
                const float v = -p.vmax + 2.f * p.vmax * (float)k / (float)(p.G - 1);
                f0 = v / 8.f;
                f1 = x ? 1.f : -1.f;
                f2 = -logf(fmaxf(__ldg(p.beta + s), 1e-30f)) / 4.f;
            }
        };
        float f[4][3];
#pragma unroll
        for (int i = 0; i < 4; ++i) features(blockIdx.x, rr[i], f[i][0], f[i][1], f[i][2]);
        for (int64_t tile = blockIdx.x; tile < p.tiles && !fail; tile += gridDim.x, ++lt) {
            const int buf = (int)(lt & 1);
            // the next tile's features load while this tile is worked on
            float nf[4][3];
#pragma unroll
            for (int i = 0; i < 4; ++i) features(tile + gridDim.x, rr[i], nf[i][0], nf[i][1], nf[i][2]);
            uint64_t F[4][3];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) F[i][k] = f32x2(f[i][k], f[i][k]);
            // the accumulator buffer is free once the epilogue has read it
            // (the first use of each buffer passes at once)
            if (!mbar_wait(&accempty[buf], (((uint32_t)lt >> 1) & 1u) ^ 1u, abort_flag)) fail = true;
            for (int kc = 0; kc < nKC; ++kc, ++cc) {
                const int st = cc % kMlpStages;
                const uint32_t ph = (uint32_t)(cc / kMlpStages) & 1u;
                if (!fail && !mbar_wait(&afree[st], ph ^ 1u, abort_flag)) fail = true;
                uint8_t* a_hi = sA + st * 32768;
                uint8_t* a_lo = a_hi + 16384;
                if (!fail) {
                    uint32_t hw[4][4], lw[4][4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        // units u, u+1 (pair j): z = W1 f + b1 as one fma chain per unit
                        const int j = (kc * kMlpKC + c * 8) / 2 + e;
                        const float4 wa = sW1[2 * j], wb = sW1[2 * j + 1];
                        const uint64_t w0 = f32x2(wa.x, wa.y), w1 = f32x2(wa.z, wa.w);
                        const uint64_t w2 = f32x2(wb.x, wb.y), bb = f32x2(wb.z, wb.w);
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const uint64_t z = fma_f32x2(w2, F[i][2], fma_f32x2(w1, F[i][1], fma_f32x2(w0, F[i][0], bb)));
                            const float h0 = fmaxf(lo_f32(z), 0.f), h1 = fmaxf(hi_f32(z), 0.f);
                            hw[i][e] = pack_bf16x2(h0, h1);
                            // the bf16 pair back in float32: its bits are the high halves
                            const uint64_t d = sub_f32x2(f32x2(h0, h1),
                                                         f32x2(__uint_as_float(hw[i][e] << 16),
                                                               __uint_as_float(hw[i][e] & 0xFFFF0000u)));
                            lw[i][e] = pack_bf16x2(lo_f32(d), hi_f32(d));
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = rr[i];
                        const int off = (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4);
                        *reinterpret_cast<uint4*>(a_hi + off) = make_uint4(hw[i][0], hw[i][1], hw[i][2], hw[i][3]);
                        *reinterpret_cast<uint4*>(a_lo + off) = make_uint4(lw[i][0], lw[i][1], lw[i][2], lw[i][3]);
                    }
                }
                fence_proxy_async_smem();
                // all producer threads agree on going on
                if (bar_sync_or(1, kMlpProducers, fail || *abort_flag)) {
                    fail = true;
                    break;
                }
                if (threadIdx.x == 128) {
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)buf * bstride;
                    const uint64_t bd = sw128_desc(smem_u32(sB + (size_t)kc * H * 128));
#pragma unroll
                    for (int pl = 0; pl < 2; ++pl) {
                        const uint64_t ad = sw128_desc(smem_u32(a_hi + pl * 16384));
#pragma unroll
                        for (int ks = 0; ks < kMlpKC / 16; ++ks)
                            tc_mma(d, ad + 2 * ks, bd + 2 * ks, idesc, (kc | pl | ks) != 0 ? 1u : 0u);
                    }
                    tc_commit(&afree[st]);
                    if (kc == nKC - 1) tc_commit(&accfull[buf]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) f[i][k] = nf[i][k];
        }
        if (fail && threadIdx.x == 128) set_abort(abort_flag, p.status);
    } else {
        // ---- epilogue: thread = TMEM lane = row of the tile
        const int quad = warp;
        int64_t lt = 0;
        for (int64_t tile = blockIdx.x; tile < p.tiles; tile += gridDim.x, ++lt) {
            const int buf = (int)(lt & 1);
            const bool ok =
                __all_sync(0xffffffffu, mbar_wait(&accfull[buf], ((uint32_t)lt >> 1) & 1u, abort_flag));
            if (!ok) {
                if (lane == 0) set_abort(abort_flag, p.status);
                break;
            }
            tc_fence_after();
            const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)buf * bstride;
            uint64_t s01 = 0, s23 = 0;       // four partial sums (columns mod 4), as pairs
#pragma unroll 1
            for (int ch = 0; ch < H / 32; ch += 2) {        // H / 32 is even
                uint32_t v[64];
                tmem_ld32(tbase + (uint32_t)(ch * 32), *reinterpret_cast<uint32_t(*)[32]>(v));
                tmem_ld32(tbase + (uint32_t)(ch * 32 + 32), *reinterpret_cast<uint32_t(*)[32]>(v + 32));
                tmem_ld_wait();
#pragma unroll
                for (int t = 0; t < 64; t += 4) {
                    const int col = ch * 32 + t;
                    const float4 a = sBW[col / 2], b = sBW[col / 2 + 1];
                    const uint64_t z01 = add_f32x2(f32x2(__uint_as_float(v[t]), __uint_as_float(v[t + 1])),
                                                   f32x2(a.x, a.y));
                    const uint64_t z23 = add_f32x2(f32x2(__uint_as_float(v[t + 2]), __uint_as_float(v[t + 3])),
                                                   f32x2(b.x, b.y));
                    s01 = fma_f32x2(f32x2(a.z, a.w), f32x2(fmaxf(lo_f32(z01), 0.f), fmaxf(hi_f32(z01), 0.f)), s01);
                    s23 = fma_f32x2(f32x2(b.z, b.w), f32x2(fmaxf(lo_f32(z23), 0.f), fmaxf(hi_f32(z23), 0.f)), s23);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[buf]);
            const int64_t row = tile * kMlpM + quad * 32 + lane;
            if (row < p.n)
                p.out[row] = __fadd_rn(__fadd_rn(__fadd_rn(lo_f32(s01), hi_f32(s01)), __fadd_rn(lo_f32(s23), hi_f32(s23))), b3);
        }
    }

    // teardown: every MMA this CTA issued has completed before TMEM is freed
    __syncthreads();
    if (threadIdx.x == 128) {
        tc_commit(done);
        (void)mbar_wait(done, 0u, never_set);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

bool mlp_tc_supported(int H)
{
    return H >= 64 && H <= 256 && H % kMlpKC == 0;
}

cudaError_t launch_mlp_forward_tc(const float* w, int H, int64_t n, const float* F, const float* beta, int G,
                                  float vmax, float* out, int* status, cudaStream_t st)
{
    if (!mlp_tc_supported(H)) return cudaErrorNotSupported;
    if (n <= 0) return cudaSuccess;
    MlpTcParams p;
    p.w = w;
    p.H = H;
    p.n = n;
    p.tiles = (n + kMlpM - 1) / kMlpM;
    p.F = F;
    p.beta = beta;
    p.G = G;
    p.vmax = vmax;
    p.out = out;
    p.status = status;
    const size_t smem = mlp_tc_smem_bytes(H);
    cudaError_t e = cudaFuncSetAttribute(mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_forward_tc_kernel, kMlpThreads, smem)) !=
        cudaSuccess)
        return e;
    // resident CTAs share the SM's 512 TMEM columns
    per_sm = std::max(1, std::min(per_sm, (int)(512 / tmem_cols_for(H))));
    const int64_t grid = std::min<int64_t>(p.tiles, (int64_t)sms * per_sm);
    mlp_forward_tc_kernel<<<(unsigned)grid, kMlpThreads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace hobo
