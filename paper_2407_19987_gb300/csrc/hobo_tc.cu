// tcgen05 tensor-core contraction of dense order-3 instances.
//
// For a tile of 128 states and a variable m the kernel forms, on the tensor
// cores, D[b][j] = sum_l x_bl * S3[m][j][l]: the tensor reshaped to
// (N^2 x N) rows (m, j) against the bit matrix, which is the first step of
// the one-index-at-a-time contraction order (Sec. VI.B / VI.F, Sec. IV.C for
// the batch).  The 0/1 state bits are exact in bf16; each cubic coefficient
// is split into 2 or 3 bf16 planes (hi + lo [+ mid]) whose products
// accumulate in float32 in tensor memory.  The fused epilogue finishes the
// contraction on CUDA cores:
//   c_bm = 1/2 sum_j x_bj D[b][j]      (cubic part of the field g_bm)
//   q_bm = sum_j x_bj S2[m][j]         (quadratic part)
//   g_bm = a_m + q_bm + c_bm
// and the energy by Euler's identity per degree,
//   E_b = sum_m x_bm a_m + 1/2 sum_m x_bm q_bm + 1/6 sum_m x_bm (2 c_bm).
//
// Roles (192 threads): warp 0 issues TMA loads of the coefficient slabs
// (128-byte swizzle, 5-stage ring), warp 1 issues the MMAs (one thread),
// warps 2-5 read the accumulators (double-buffered, 2 x 256 columns) and
// run the epilogue; the quadratic parts q_bm come from a small pre-pass
// (pair_fields_kernel).  All threads expand the state bits of a tile into the
// bf16 A operand in shared memory.  CTA c owns state tile c % T and a chunk
// of the variables m; tiles advance through m in step.  Every wait on an mbarrier gives up
// after kWaitNs and reports HOBO_ERR_TIMEOUT through the status word.
#include <algorithm>
#include <vector>
#include <cuda.h>
#include "hobo_internal.h"
#include "hobo_dev.cuh"
#include "tc_common.cuh"

namespace hobo {

constexpr int kTcM = 128;          // states per tile (MMA M)
constexpr int kTcKB = 64;          // K elements per swizzle atom (128 bytes)
constexpr int kTcStages = 5;
constexpr int kTcThreads = 192;

struct TcParams {
    const uint32_t* X;
    int B, N, W, NJ, KP, nsplit, P;
    const float* Qt;     // [N][B] quadratic parts q_bm, from pair_fields_kernel
    const float* a;
    float* out_g;
    int flip;
    float* Epart;        // [G][128][4]
    int T, chunks, G;    // state tiles, m-chunks per tile, CTAs (= T * chunks)
    int* status;
};

__global__ void __launch_bounds__(kTcThreads, 1)
energy_tc_kernel(const __grid_constant__ CUtensorMap tmap, const TcParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int nKB = p.KP / kTcKB;
    const uint32_t stage_bytes = (uint32_t)p.NJ * 128u;
    uint8_t* sA = smem;                                  // nKB x 16 KB
    uint8_t* sB = sA + nKB * 16384;                      // kTcStages x stage_bytes
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kTcStages * stage_bytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + kTcStages;
    uint64_t* afull = bars + 2 * kTcStages;
    uint64_t* aempty = afull + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(aempty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    volatile int* never_set = abort_flag + 1;     // stays 0: teardown waits use only the time limit

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = p.N, W = p.W, B = p.B;
    const int c = blockIdx.x;
    // CTA c: state tile c % T, variables m in chunk c / T.  All tiles walk
    // the same m at the same time, so each coefficient slab is fetched from
    // memory once and served to the other tiles from L2.
    const int tile_c = c % p.T, chunk = c / p.T;
    const int i0 = tile_c * N + (int)((int64_t)chunk * N / p.chunks);
    const int i1 = tile_c * N + (int)((int64_t)(chunk + 1) * N / p.chunks);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&afull[s], 1);
            mbar_init(&aempty[s], 4);
        }
        *abort_flag = 0;
        *never_set = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    // role state carried across segments
    int pstage = 0;
    uint32_t pphase = 0;                 // producer ring position
    uint32_t armed_phase[kTcStages];     // last phase the producer armed per stage
    bool armed[kTcStages];
    for (int s = 0; s < kTcStages; ++s) { armed[s] = false; armed_phase[s] = 0; }
    int cstage = 0;
    uint32_t cphase = 0;                 // MMA ring position
    int acc_mma = 0, acc_epi = 0;        // accumulator counters (buffer = n & 1)
    const uint32_t idesc = idesc_bf16(kTcM, p.NJ);

    int seg = 0;
    for (int it = i0; it < i1; ++seg) {
        const int tile = it / N;
        const int seg_end = min(i1, (tile + 1) * N);

        // ---- A operand: bits of the tile's 128 states as bf16 0/1, K-major,
        // 128-byte swizzle (16-byte chunk c of row r stored at c ^ (r & 7)).
        {
            const int cpr = p.KP / 8;     // 16-byte chunks per row
            for (int q = threadIdx.x; q < kTcM * cpr; q += blockDim.x) {
                const int r = q / cpr, cc = q % cpr;
                const int kb = cc >> 3, ch = cc & 7;
                const int b = tile * kTcM + r;
                const int l0 = cc * 8;
                uint32_t byte = 0;
                if (b < B && l0 < N) {
                    byte = (p.X[(int64_t)b * W + (l0 >> 5)] >> (l0 & 31)) & 0xFFu;
                    const int rem = N - l0;
                    if (rem < 8) byte &= (1u << rem) - 1u;
                }
                uint32_t wv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t lo = ((byte >> (2 * e)) & 1u) ? 0x3F80u : 0u;
                    const uint32_t hi = ((byte >> (2 * e + 1)) & 1u) ? 0x3F80u : 0u;
                    wv[e] = lo | (hi << 16);
                }
                uint8_t* dst = sA + kb * 16384 + (r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4);
                *reinterpret_cast<uint4*>(dst) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();

        if (warp == 0) {
            if (lane == 0) {
                // ---- producer: coefficient slabs of planes q for items m
                for (int j = it; j < seg_end && !*abort_flag; ++j) {
                    const int m = j % N;
                    for (int q = 0; q < p.nsplit; ++q)
                        for (int kb = 0; kb < nKB; ++kb) {
                            if (!mbar_wait(&empty[pstage], pphase ^ 1u, abort_flag)) {
                                set_abort(abort_flag, p.status);
                                break;
                            }
                            mbar_expect_tx(&full[pstage], stage_bytes);
                            tma_load_2d(sB + pstage * stage_bytes, &tmap, kb * kTcKB, (q * N + m) * p.NJ,
                                        &full[pstage]);
                            armed[pstage] = true;
                            armed_phase[pstage] = pphase;
                            if (++pstage == kTcStages) { pstage = 0; pphase ^= 1u; }
                        }
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {
                // ---- MMA issuer
                for (int j = it; j < seg_end && !*abort_flag; ++j) {
                    const int buf = acc_mma & 1;
                    if (!mbar_wait(&aempty[buf], (((uint32_t)acc_mma >> 1) & 1u) ^ 1u, abort_flag)) {
                        set_abort(abort_flag, p.status);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(buf * 256);
                    uint32_t accum = 0;
                    bool ok = true;
                    for (int q = 0; q < p.nsplit && ok; ++q)
                        for (int kb = 0; kb < nKB; ++kb) {
                            if (!mbar_wait(&full[cstage], cphase, abort_flag)) {
                                set_abort(abort_flag, p.status);
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint64_t ad = sw128_desc(smem_u32(sA + kb * 16384));
                            const uint64_t bd = sw128_desc(smem_u32(sB + cstage * stage_bytes));
#pragma unroll
                            for (int k = 0; k < kTcKB / 16; ++k) {
                                tc_mma(d, ad + 2 * k, bd + 2 * k, idesc, accum);
                                accum = 1;
                            }
                            tc_commit(&empty[cstage]);
                            if (++cstage == kTcStages) { cstage = 0; cphase ^= 1u; }
                        }
                    if (!ok) break;
                    tc_commit(&afull[buf]);
                    ++acc_mma;
                }
            }
        } else {
            // ---- epilogue: thread = TMEM lane = state row
            const int quad = warp & 3;
            const int r = quad * 32 + lane;
            const int b = tile * kTcM + r;
            uint32_t x[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                uint32_t v = (b < B && k < W) ? p.X[(int64_t)b * W + k] : 0u;
                const int rem = N - 32 * k;
                if (rem <= 0) v = 0u; else if (rem < 32) v &= (1u << rem) - 1u;
                x[k] = v;
            }
            float e1 = 0.f, e2 = 0.f, e3 = 0.f;
            const int nch = (p.NJ + 31) / 32;   // columns >= N meet zero bits
            for (int j = it; j < seg_end; ++j) {
                const int m = j % N;
                const int buf = acc_epi & 1;
                // quadratic part, from the pair pre-pass
                const float q = b < B ? __ldg(p.Qt + (int64_t)m * B + b) : 0.f;
                // the warp leaves together: tcgen05.ld below needs all 32 lanes
                const bool ok = __all_sync(0xffffffffu, mbar_wait(&afull[buf], ((uint32_t)acc_epi >> 1) & 1u, abort_flag));
                if (!ok) {
                    if (lane == 0) set_abort(abort_flag, p.status);
                    break;
                }
                tc_fence_after();
                float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
                const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 256);
                uint32_t xr[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) xr[k] = x[k];
#pragma unroll 1
                for (int ch = 0; ch < nch; ++ch) {
                    uint32_t v[32];
                    tmem_ld32(tbase + (uint32_t)(ch * 32), v);
                    tmem_ld_wait();
                    const uint32_t xw = xr[0];
#pragma unroll
                    for (int k = 0; k < 7; ++k) xr[k] = xr[k + 1];
                    // add the accumulator of column j where bit j is set (the
                    // same value as x * D + c with x in {0, 1})
#pragma unroll
                    for (int t = 0; t < 32; t += 4) {
                        if ((xw >> t) & 1u) c0 = __fadd_rn(c0, __uint_as_float(v[t]));
                        if ((xw >> (t + 1)) & 1u) c1 = __fadd_rn(c1, __uint_as_float(v[t + 1]));
                        if ((xw >> (t + 2)) & 1u) c2 = __fadd_rn(c2, __uint_as_float(v[t + 2]));
                        if ((xw >> (t + 3)) & 1u) c3 = __fadd_rn(c3, __uint_as_float(v[t + 3]));
                    }
                }
                const float cacc = __fadd_rn(__fadd_rn(c0, c1), __fadd_rn(c2, c3));
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&aempty[buf]);
                ++acc_epi;
                const float am = __ldg(p.a + m);
                const float g = __fadd_rn(__fadd_rn(am, q), __fmul_rn(0.5f, cacc));
                uint32_t xmw = x[0];
#pragma unroll
                for (int k = 1; k < 8; ++k) xmw = ((m >> 5) == k) ? x[k] : xmw;
                const bool xm = (xmw >> (m & 31)) & 1u;
                if (xm) {
                    e1 = __fadd_rn(e1, am);
                    e2 = __fadd_rn(e2, q);
                    e3 = __fadd_rn(e3, cacc);
                }
                if (b < B && p.out_g) p.out_g[(int64_t)b * N + m] = (p.flip && xm) ? -g : g;
            }
            float* dst = p.Epart + ((int64_t)c * kTcM + r) * 4;
            dst[0] = e1; dst[1] = e2; dst[2] = e3; dst[3] = 0.f;
        }
        __syncthreads();
        it = seg_end;
    }

    // teardown: make sure no TMA copy is still landing in shared memory
    if (warp == 0 && lane == 0 && *abort_flag) {
        for (int s = 0; s < kTcStages; ++s)
            if (armed[s]) (void)mbar_wait(&full[s], armed_phase[s], never_set);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// Quadratic parts of the fields for the tensor-core epilogue:
// Qt[m][b] = q_bm = sum_j x_bj S2[m][j], as four partial sums over the
// columns j = 4t + u (u = 0..3), added (0 + 1) + (2 + 3).  A block takes 128
// states (one per thread) and a chunk of rows m, staged in shared memory.
constexpr int kPairThreads = 128;

__global__ void __launch_bounds__(kPairThreads)
pair_fields_kernel(const uint32_t* __restrict__ X, int B, int N, int W, const float* __restrict__ S2, int P,
                   int mchunk, float* __restrict__ Qt)
{
    __shared__ float4 row[64];
    const int b = blockIdx.x * kPairThreads + threadIdx.x;
    uint32_t x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        uint32_t v = (b < B && k < W) ? X[(int64_t)b * W + k] : 0u;
        const int rem = N - 32 * k;
        if (rem <= 0) v = 0u; else if (rem < 32) v &= (1u << rem) - 1u;
        x[k] = v;
    }
    const int P4 = P >> 2;
    const int m0 = blockIdx.y * mchunk, m1 = min(N, m0 + mchunk);
    for (int m = m0; m < m1; ++m) {
        __syncthreads();
        if (threadIdx.x < P4) row[threadIdx.x] = __ldg(reinterpret_cast<const float4*>(S2 + (int64_t)m * P) + threadIdx.x);
        __syncthreads();
        float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f;
        uint32_t xr[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) xr[k] = x[k];
#pragma unroll 1
        for (int k = 0; k < 8; ++k) {
            if (8 * k >= P4) break;
            const uint32_t xw = xr[0];
#pragma unroll
            for (int k2 = 0; k2 < 7; ++k2) xr[k2] = xr[k2 + 1];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                if (8 * k + t >= P4) break;
                const float4 v = row[8 * k + t];
                q0 = fmaf((float)((xw >> (4 * t)) & 1u), v.x, q0);
                q1 = fmaf((float)((xw >> (4 * t + 1)) & 1u), v.y, q1);
                q2 = fmaf((float)((xw >> (4 * t + 2)) & 1u), v.z, q2);
                q3 = fmaf((float)((xw >> (4 * t + 3)) & 1u), v.w, q3);
            }
        }
        if (b < B) Qt[(int64_t)m * B + b] = __fadd_rn(__fadd_rn(q0, q1), __fadd_rn(q2, q3));
    }
}

// Timeout self-test: one thread waits, through the same bounded wait as the
// contraction kernel, on an mbarrier that nothing arrives at; when the
// limit runs out it records the timeout in the instance's status word the
// way the contraction kernel does.
__global__ void wait_timeout_selftest_kernel(int* status, uint64_t limit_ns)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0u, &abort_flag, limit_ns)) set_abort(&abort_flag, status);
}

cudaError_t launch_wait_timeout_selftest(const hobo_instance* h, uint64_t limit_ns, cudaStream_t st)
{
    wait_timeout_selftest_kernel<<<1, 32, 0, st>>>(h->status, limit_ns);
    return cudaGetLastError();
}

// E_b from the partial sums of the m-chunks of its tile, added in chunk
// order: E = sum x_m a_m + 1/2 sum x_m q_m + 1/6 sum x_m (2 c_m).
__global__ void energy_tc_finalize(const float* __restrict__ Epart, int B, int T, int chunks,
                                   float* __restrict__ E)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int t = b / kTcM, r = b % kTcM;
    float s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int k = 0; k < chunks; ++k) {
        const float* src = Epart + ((int64_t)(k * T + t) * kTcM + r) * 4;
        s1 = __fadd_rn(s1, src[0]);
        s2 = __fadd_rn(s2, src[1]);
        s3 = __fadd_rn(s3, src[2]);
    }
    E[b] = __fadd_rn(__fadd_rn(s1, __fmul_rn(0.5f, s2)), __fdiv_rn(s3, 6.0f));
}

static size_t tc_smem_bytes(int NJ, int KP)
{
    return 1024 + (size_t)(KP / kTcKB) * 16384 + (size_t)kTcStages * NJ * 128 + 256;
}

bool tc_supported(const hobo_instance* h)
{
    return h->dense && h->d.S3bf && h->d.tmap_ok && h->N <= 256;
}

static cudaError_t encode_planes_map(void* map_out, const void* base, int planes, int N, int NJ, int KP,
                                     int box_rows)
{
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)KP, (cuuint64_t)planes * N * NJ};
    cuuint64_t strides[1] = {(cuuint64_t)KP * 2};
    cuuint32_t box[2] = {(cuuint32_t)kTcKB, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = reinterpret_cast<EncodeFn>(fn)(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                                                2, const_cast<void*>(base), dims, strides, box, estr,
                                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_tc_tensor_map(hobo_instance* h)
{
    const auto& d = h->d;
    cudaError_t e = encode_planes_map(h->d.tmap, d.S3bf, d.nsplit, h->N, d.NJ, d.KP, d.NJ);
    h->d.tmap_ok = e == cudaSuccess;
    return e;
}

cudaError_t make_tc_tensor_map_rs(hobo_instance* h)
{
    const auto& d = h->d;
    cudaError_t e = encode_planes_map(h->d.tmap_rs, d.S3limb, d.rs_L, h->N, d.NJ, d.KP, d.NJ);
    h->d.tmap_rs_ok = e == cudaSuccess;
    return e;
}

// ---------------------------------------------------------------------------
// Order-4 tensor-core contraction: the symmetric quartic tensor reshaped to
// (N^3 x N) rows (m, j, k), K = l, against the bit matrix (the next index of
// the one-at-a-time contraction order of Sec. VI).  Items are (m, chunk of
// 256 rows (j, k)); the epilogue adds the accumulators of rows whose bits
// j and k are both set: c_bm = sum_{j,k,l} S4[m][j][k][l] x_j x_k x_l =
// 6 g4_bm (the quartic part of the field), and sum_m x_bm c_bm = 24 E4.
// Same roles, stages and bounded waits as the order-3 kernel.
// ---------------------------------------------------------------------------
struct Tc4Params {
    const uint32_t* X;
    int B, N, W, R4, nsplit;
    int T, chunks, G;
    float* G4;        // [B][N] quartic field parts
    float* Epart;     // [G][128][4]
    int* status;
};

__global__ void __launch_bounds__(kTcThreads, 1)
energy_tc4_kernel(const __grid_constant__ CUtensorMap tmap, const Tc4Params p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int NJ4 = 256;
    const uint32_t stage_bytes = (uint32_t)NJ4 * 128u;
    uint8_t* sA = smem;                          // one K block (l < 64)
    uint8_t* sB = sA + 16384;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kTcStages * stage_bytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + kTcStages;
    uint64_t* afull = bars + 2 * kTcStages;
    uint64_t* aempty = afull + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(aempty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    volatile int* never_set = abort_flag + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = p.N, W = p.W, B = p.B;
    const int nch4 = p.R4 / NJ4;                 // row chunks per m
    const int c = blockIdx.x;
    const int tile_c = c % p.T, chunk = c / p.T;
    const int i0 = tile_c * N + (int)((int64_t)chunk * N / p.chunks);
    const int i1 = tile_c * N + (int)((int64_t)(chunk + 1) * N / p.chunks);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&afull[s], 1);
            mbar_init(&aempty[s], 4);
        }
        *abort_flag = 0;
        *never_set = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    int pstage = 0;
    uint32_t pphase = 0;
    uint32_t armed_phase[kTcStages];
    bool armed[kTcStages];
    for (int s = 0; s < kTcStages; ++s) { armed[s] = false; armed_phase[s] = 0; }
    int cstage = 0;
    uint32_t cphase = 0;
    int acc_mma = 0, acc_epi = 0;
    const uint32_t idesc = idesc_bf16(kTcM, NJ4);

    int seg = 0;
    for (int it = i0; it < i1; ++seg) {
        const int tile = it / N;
        const int seg_end = min(i1, (tile + 1) * N);
        // A operand: bits l < 64 of the tile's 128 states, bf16, swizzled
        for (int q = threadIdx.x; q < kTcM * 8; q += blockDim.x) {
            const int r = q >> 3, ch = q & 7;
            const int b = tile * kTcM + r;
            const int l0 = ch * 8;
            uint32_t byte = 0;
            if (b < B && l0 < N) {
                byte = (p.X[(int64_t)b * W + (l0 >> 5)] >> (l0 & 31)) & 0xFFu;
                const int rem = N - l0;
                if (rem < 8) byte &= (1u << rem) - 1u;
            }
            uint32_t wv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t lo = ((byte >> (2 * e)) & 1u) ? 0x3F80u : 0u;
                const uint32_t hi = ((byte >> (2 * e + 1)) & 1u) ? 0x3F80u : 0u;
                wv[e] = lo | (hi << 16);
            }
            uint8_t* dst = sA + (r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4);
            *reinterpret_cast<uint4*>(dst) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        fence_proxy_async_smem();
        __syncthreads();

        if (warp == 0) {
            if (lane == 0) {
                for (int j = it; j < seg_end && !*abort_flag; ++j) {
                    const int m = j % N;
                    for (int cc = 0; cc < nch4; ++cc)
                        for (int q = 0; q < p.nsplit; ++q) {
                            if (!mbar_wait(&empty[pstage], pphase ^ 1u, abort_flag)) {
                                set_abort(abort_flag, p.status);
                                break;
                            }
                            mbar_expect_tx(&full[pstage], stage_bytes);
                            tma_load_2d(sB + pstage * stage_bytes, &tmap, 0, (q * N + m) * p.R4 + cc * NJ4,
                                        &full[pstage]);
                            armed[pstage] = true;
                            armed_phase[pstage] = pphase;
                            if (++pstage == kTcStages) { pstage = 0; pphase ^= 1u; }
                        }
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {
                bool ok = true;
                for (int j = it; j < seg_end && ok && !*abort_flag; ++j) {
                    for (int cc = 0; cc < nch4 && ok; ++cc) {
                        const int buf = acc_mma & 1;
                        if (!mbar_wait(&aempty[buf], (((uint32_t)acc_mma >> 1) & 1u) ^ 1u, abort_flag)) {
                            set_abort(abort_flag, p.status);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d = tmem + (uint32_t)(buf * 256);
                        uint32_t accum = 0;
                        for (int q = 0; q < p.nsplit; ++q) {
                            if (!mbar_wait(&full[cstage], cphase, abort_flag)) {
                                set_abort(abort_flag, p.status);
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint64_t ad = sw128_desc(smem_u32(sA));
                            const uint64_t bd = sw128_desc(smem_u32(sB + cstage * stage_bytes));
#pragma unroll
                            for (int k = 0; k < kTcKB / 16; ++k) {
                                tc_mma(d, ad + 2 * k, bd + 2 * k, idesc, accum);
                                accum = 1;
                            }
                            tc_commit(&empty[cstage]);
                            if (++cstage == kTcStages) { cstage = 0; cphase ^= 1u; }
                        }
                        if (!ok) break;
                        tc_commit(&afull[buf]);
                        ++acc_mma;
                    }
                }
            }
        } else {
            const int quad = warp & 3;
            const int r = quad * 32 + lane;
            const int b = tile * kTcM + r;
            uint32_t x[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                uint32_t v = (b < B && k < W) ? p.X[(int64_t)b * W + k] : 0u;
                const int rem = N - 32 * k;
                if (rem <= 0) v = 0u; else if (rem < 32) v &= (1u << rem) - 1u;
                x[k] = v;
            }
            float e4 = 0.f;
            bool ok = true;
            for (int j = it; j < seg_end && ok; ++j) {
                const int m = j % N;
                float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
                for (int cc = 0; cc < nch4; ++cc) {
                    const int buf = acc_epi & 1;
                    ok = __all_sync(0xffffffffu, mbar_wait(&afull[buf], ((uint32_t)acc_epi >> 1) & 1u, abort_flag));
                    if (!ok) {
                        if (lane == 0) set_abort(abort_flag, p.status);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 256);
#pragma unroll 1
                    for (int g = 0; g < 8; ++g) {
                        // columns 32g..32g+31 of chunk cc: row = cc*256 + 32g + t,
                        // j = row / 64 (fixed in the group), k = (g & 1) * 32 + t
                        const int jj = (cc * NJ4 + 32 * g) >> 6;
                        const uint32_t xj = jj < 32 ? (x[0] >> jj) & 1u : (x[1] >> (jj - 32)) & 1u;
                        const uint32_t xw = xj ? x[g & 1] : 0u;
                        if (!__any_sync(0xffffffffu, xw != 0u)) continue;
                        uint32_t v[32];
                        tmem_ld32(tbase + (uint32_t)(g * 32), v);
                        tmem_ld_wait();
#pragma unroll
                        for (int t = 0; t < 32; t += 4) {
                            if ((xw >> t) & 1u) c0 = __fadd_rn(c0, __uint_as_float(v[t]));
                            if ((xw >> (t + 1)) & 1u) c1 = __fadd_rn(c1, __uint_as_float(v[t + 1]));
                            if ((xw >> (t + 2)) & 1u) c2 = __fadd_rn(c2, __uint_as_float(v[t + 2]));
                            if ((xw >> (t + 3)) & 1u) c3 = __fadd_rn(c3, __uint_as_float(v[t + 3]));
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&aempty[buf]);
                    ++acc_epi;
                }
                if (!ok) break;
                const float cm = __fadd_rn(__fadd_rn(c0, c1), __fadd_rn(c2, c3));
                const bool xm = ((m < 32 ? x[0] >> m : x[1] >> (m - 32)) & 1u) != 0u;
                if (xm) e4 = __fadd_rn(e4, cm);
                if (b < B) p.G4[(int64_t)b * N + m] = __fdiv_rn(cm, 6.0f);
            }
            float* dst = p.Epart + (((int64_t)c) * kTcM + r) * 4;
            dst[0] = e4; dst[1] = 0.f; dst[2] = 0.f; dst[3] = 0.f;
        }
        __syncthreads();
        it = seg_end;
    }

    if (warp == 0 && lane == 0 && *abort_flag) {
        for (int s = 0; s < kTcStages; ++s)
            if (armed[s]) (void)mbar_wait(&full[s], armed_phase[s], never_set);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// E = E_low + (1/24) sum of the quartic partials of the tile's m-chunks (in
// chunk order); g = g_low + g4 (g_low already in g when there is a lower
// part), with dE = (1 - 2 x) g when flip.
__global__ void energy_tc4_finalize(const float* __restrict__ Epart, const float* __restrict__ G4,
                                    const uint32_t* __restrict__ X, int B, int N, int W, int T, int chunks,
                                    int has_low, int flip, float* __restrict__ E, float* __restrict__ g)
{
    const int b = blockIdx.x;
    if (b >= B) return;
    const int t = b / kTcM, r = b % kTcM;
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int k = 0; k < chunks; ++k) s = __fadd_rn(s, Epart[((int64_t)(k * T + t) * kTcM + r) * 4]);
        const float e4 = __fdiv_rn(s, 24.0f);
        E[b] = has_low ? __fadd_rn(E[b], e4) : e4;
    }
    if (g) {
        for (int m = threadIdx.x; m < N; m += blockDim.x) {
            const int64_t at = (int64_t)b * N + m;
            float v = has_low ? __fadd_rn(g[at], G4[at]) : G4[at];
            if (flip && ((X[(int64_t)b * W + (m >> 5)] >> (m & 31)) & 1u)) v = -v;
            g[at] = v;
        }
    }
}

bool tc4_supported(const hobo_instance* h)
{
    return h->order == 4 && h->d.S4bf && h->d.tmap4_ok && h->N <= 64;
}

cudaError_t make_tc4_tensor_map(hobo_instance* h)
{
    const auto& d = h->d;
    cudaError_t e = encode_planes_map(h->d.tmap4, d.S4bf, d.nsplit4, h->N, d.R4, 64, 256);
    h->d.tmap4_ok = e == cudaSuccess;
    return e;
}

cudaError_t launch_energy_tc4(const hobo_instance* h, const uint32_t* X, int B, float* E, float* g_or_dE,
                              bool flip_out, cudaStream_t st)
{
    if (!tc4_supported(h)) return cudaErrorNotSupported;
    if (B == 0) return cudaSuccess;
    const auto& d = h->d;
    cudaError_t e = cudaSuccess;
    if (h->low) e = launch_energy_terms(h->low, X, B, E, g_or_dE, false, st);
    if (e != cudaSuccess) return e;
    const int tiles = (B + kTcM - 1) / kTcM;
    const int chunks = std::max(1, std::min(h->N, h->num_sms / tiles));
    Tc4Params p{};
    p.X = X; p.B = B; p.N = h->N; p.W = h->W; p.R4 = d.R4; p.nsplit = d.nsplit4;
    p.T = tiles; p.chunks = chunks; p.G = tiles * chunks; p.status = h->status;
    float *Epart = nullptr, *G4 = nullptr;
    e = cudaMallocAsync((void**)&Epart, sizeof(float) * (size_t)p.G * kTcM * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&G4, sizeof(float) * (size_t)B * h->N, st);
    p.Epart = Epart;
    p.G4 = G4;
    const size_t sm = 1024 + 16384 + (size_t)kTcStages * 256 * 128 + 256;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(energy_tc4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) {
        const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(d.tmap4);
        energy_tc4_kernel<<<p.G, kTcThreads, sm, st>>>(*map, p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        energy_tc4_finalize<<<B, 64, 0, st>>>(Epart, G4, X, B, h->N, h->W, tiles, chunks, h->low ? 1 : 0,
                                              flip_out ? 1 : 0, E, g_or_dE);
        e = cudaGetLastError();
    }
    if (Epart) cudaFreeAsync(Epart, st);
    if (G4) cudaFreeAsync(G4, st);
    return e;
}

// ---------------------------------------------------------------------------
// Order-k tensor-core contraction, k = 5 or 6 (the order-4 kernel's scheme
// with rows over sorted index prefixes).  The top-degree part of the field
// of m is g_m = sum over (k-1)-sets T not containing m of c_{T+m} x^T.  Each
// T is split into its k-2 smallest members P (a sorted prefix) and its
// largest member l, so with rows (m, P) over every sorted (k-2)-subset P of
// the variables and K = l,
//   D[b][(m, P)] = sum_{l > max P} C[m][P][l] x_bl
// on the tensor cores, and g_bm = sum over rows whose prefix bits are all set
// of D (each T once: no (k-1)! repeats of a fully symmetric tensor).  The
// energy takes the rows with min P > m only (each monomial once, at its
// smallest member m): E_k = sum_m x_bm sum_{P > m, x^P = 1} D.  Each row's
// prefix is a bit mask (N <= 64) and its smallest member, in tables read by
// the epilogue.  Coefficients split into bf16 planes (hi + lo, exact for
// integers below 2^16; hi + mid + lo otherwise), float32 accumulation.  Same
// roles, stages and bounded waits as the order-4 kernel; items are (m,
// 256-row chunk).
// ---------------------------------------------------------------------------
struct TckParams {
    const uint32_t* X;
    int B, N, W, RK, nsplit;
    int T, chunks, G;
    const unsigned long long* rmask;   // [RK] prefix bits of each row (padding rows: 0, zero planes)
    const uint8_t* rmin;               // [RK] smallest member of the prefix
    float* GK;        // [B][N] top-degree field parts
    float* Epart;     // [G][128][4]
    int* status;
};

__global__ void __launch_bounds__(kTcThreads, 1)
energy_tck_kernel(const __grid_constant__ CUtensorMap tmap, const TckParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int NJK = 256;
    const uint32_t stage_bytes = (uint32_t)NJK * 128u;
    uint8_t* sA = smem;                          // one K block (l < 64)
    uint8_t* sB = sA + 16384;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kTcStages * stage_bytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + kTcStages;
    uint64_t* afull = bars + 2 * kTcStages;
    uint64_t* aempty = afull + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(aempty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    volatile int* never_set = abort_flag + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = p.N, W = p.W, B = p.B;
    const int nchk = p.RK / NJK;                 // row chunks per m
    const int c = blockIdx.x;
    const int tile_c = c % p.T, chunk = c / p.T;
    const int i0 = tile_c * N + (int)((int64_t)chunk * N / p.chunks);
    const int i1 = tile_c * N + (int)((int64_t)(chunk + 1) * N / p.chunks);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&afull[s], 1);
            mbar_init(&aempty[s], 4);
        }
        *abort_flag = 0;
        *never_set = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    int pstage = 0;
    uint32_t pphase = 0;
    uint32_t armed_phase[kTcStages];
    bool armed[kTcStages];
    for (int s = 0; s < kTcStages; ++s) { armed[s] = false; armed_phase[s] = 0; }
    int cstage = 0;
    uint32_t cphase = 0;
    int acc_mma = 0, acc_epi = 0;
    const uint32_t idesc = idesc_bf16(kTcM, NJK);

    for (int it = i0; it < i1;) {
        const int tile = it / N;
        const int seg_end = min(i1, (tile + 1) * N);
        // A operand: bits l < 64 of the tile's 128 states, bf16, swizzled
        for (int q = threadIdx.x; q < kTcM * 8; q += blockDim.x) {
            const int r = q >> 3, ch = q & 7;
            const int b = tile * kTcM + r;
            const int l0 = ch * 8;
            uint32_t byte = 0;
            if (b < B && l0 < N) {
                byte = (p.X[(int64_t)b * W + (l0 >> 5)] >> (l0 & 31)) & 0xFFu;
                const int rem = N - l0;
                if (rem < 8) byte &= (1u << rem) - 1u;
            }
            uint32_t wv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t lo = ((byte >> (2 * e)) & 1u) ? 0x3F80u : 0u;
                const uint32_t hi = ((byte >> (2 * e + 1)) & 1u) ? 0x3F80u : 0u;
                wv[e] = lo | (hi << 16);
            }
            uint8_t* dst = sA + (r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4);
            *reinterpret_cast<uint4*>(dst) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
        fence_proxy_async_smem();
        __syncthreads();

        if (warp == 0) {
            if (lane == 0) {
                bool ok = true;
                for (int j = it; j < seg_end && ok && !*abort_flag; ++j) {
                    const int m = j % N;
                    for (int cc = 0; cc < nchk && ok; ++cc)
                        for (int q = 0; q < p.nsplit; ++q) {
                            if (!mbar_wait(&empty[pstage], pphase ^ 1u, abort_flag)) {
                                set_abort(abort_flag, p.status);
                                ok = false;
                                break;
                            }
                            mbar_expect_tx(&full[pstage], stage_bytes);
                            tma_load_2d(sB + pstage * stage_bytes, &tmap, 0, (q * N + m) * p.RK + cc * NJK,
                                        &full[pstage]);
                            armed[pstage] = true;
                            armed_phase[pstage] = pphase;
                            if (++pstage == kTcStages) { pstage = 0; pphase ^= 1u; }
                        }
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {
                bool ok = true;
                for (int j = it; j < seg_end && ok && !*abort_flag; ++j) {
                    for (int cc = 0; cc < nchk && ok; ++cc) {
                        const int buf = acc_mma & 1;
                        if (!mbar_wait(&aempty[buf], (((uint32_t)acc_mma >> 1) & 1u) ^ 1u, abort_flag)) {
                            set_abort(abort_flag, p.status);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d = tmem + (uint32_t)(buf * 256);
                        uint32_t accum = 0;
                        for (int q = 0; q < p.nsplit; ++q) {
                            if (!mbar_wait(&full[cstage], cphase, abort_flag)) {
                                set_abort(abort_flag, p.status);
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint64_t ad = sw128_desc(smem_u32(sA));
                            const uint64_t bd = sw128_desc(smem_u32(sB + cstage * stage_bytes));
#pragma unroll
                            for (int k = 0; k < kTcKB / 16; ++k) {
                                tc_mma(d, ad + 2 * k, bd + 2 * k, idesc, accum);
                                accum = 1;
                            }
                            tc_commit(&empty[cstage]);
                            if (++cstage == kTcStages) { cstage = 0; cphase ^= 1u; }
                        }
                        if (!ok) break;
                        tc_commit(&afull[buf]);
                        ++acc_mma;
                    }
                }
            }
        } else {
            const int quad = warp & 3;
            const int r = quad * 32 + lane;
            const int b = tile * kTcM + r;
            unsigned long long xb = 0ull;
            if (b < B) {
                xb = p.X[(int64_t)b * W];
                if (W > 1) xb |= (unsigned long long)p.X[(int64_t)b * W + 1] << 32;
                if (N < 64) xb &= (1ull << N) - 1ull;
            }
            float ek = 0.f;
            bool ok = true;
            for (int j = it; j < seg_end && ok; ++j) {
                const int m = j % N;
                float g0 = 0.f, g1 = 0.f, e0 = 0.f, e1 = 0.f;
                for (int cc = 0; cc < nchk; ++cc) {
                    const int buf = acc_epi & 1;
                    ok = __all_sync(0xffffffffu, mbar_wait(&afull[buf], ((uint32_t)acc_epi >> 1) & 1u, abort_flag));
                    if (!ok) {
                        if (lane == 0) set_abort(abort_flag, p.status);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 256);
#pragma unroll 1
                    for (int gq = 0; gq < 8; ++gq) {
                        uint32_t v[32];
                        tmem_ld32(tbase + (uint32_t)(gq * 32), v);
                        const int row0 = cc * NJK + 32 * gq;
                        // the 32 rows' masks and smallest members: lane t
                        // loads row t, the warp shares them by shuffles
                        const unsigned long long mk = __ldg(p.rmask + row0 + lane);
                        const int mn = __ldg(p.rmin + row0 + lane);
                        tmem_ld_wait();
#pragma unroll
                        for (int t = 0; t < 32; t += 2) {
                            const unsigned long long m0 = __shfl_sync(0xffffffffu, mk, t);
                            const unsigned long long m1 = __shfl_sync(0xffffffffu, mk, t + 1);
                            const int n0 = __shfl_sync(0xffffffffu, mn, t);
                            const int n1 = __shfl_sync(0xffffffffu, mn, t + 1);
                            if ((xb & m0) == m0) {
                                g0 = __fadd_rn(g0, __uint_as_float(v[t]));
                                if (n0 > m) e0 = __fadd_rn(e0, __uint_as_float(v[t]));
                            }
                            if ((xb & m1) == m1) {
                                g1 = __fadd_rn(g1, __uint_as_float(v[t + 1]));
                                if (n1 > m) e1 = __fadd_rn(e1, __uint_as_float(v[t + 1]));
                            }
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&aempty[buf]);
                    ++acc_epi;
                }
                if (!ok) break;
                if ((xb >> m) & 1ull) ek = __fadd_rn(ek, __fadd_rn(e0, e1));
                if (b < B) p.GK[(int64_t)b * N + m] = __fadd_rn(g0, g1);
            }
            float* dst = p.Epart + (((int64_t)c) * kTcM + r) * 4;
            dst[0] = ek; dst[1] = 0.f; dst[2] = 0.f; dst[3] = 0.f;
        }
        __syncthreads();
        it = seg_end;
    }

    if (warp == 0 && lane == 0 && *abort_flag) {
        for (int s = 0; s < kTcStages; ++s)
            if (armed[s]) (void)mbar_wait(&full[s], armed_phase[s], never_set);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// E = E_low + the top-degree partials of the tile's m-chunks (in chunk
// order); g = g_low + gK, with dE = (1 - 2 x) g when flip.
__global__ void energy_tck_finalize(const float* __restrict__ Epart, const float* __restrict__ GK,
                                    const uint32_t* __restrict__ X, int B, int N, int W, int T, int chunks,
                                    int has_low, int flip, float* __restrict__ E, float* __restrict__ g)
{
    const int b = blockIdx.x;
    if (b >= B) return;
    const int t = b / kTcM, r = b % kTcM;
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int k = 0; k < chunks; ++k) s = __fadd_rn(s, Epart[((int64_t)(k * T + t) * kTcM + r) * 4]);
        E[b] = has_low ? __fadd_rn(E[b], s) : s;
    }
    if (g) {
        for (int m = threadIdx.x; m < N; m += blockDim.x) {
            const int64_t at = (int64_t)b * N + m;
            float v = has_low ? __fadd_rn(g[at], GK[at]) : GK[at];
            if (flip && ((X[(int64_t)b * W + (m >> 5)] >> (m & 31)) & 1u)) v = -v;
            g[at] = v;
        }
    }
}

bool tck_supported(const hobo_instance* h)
{
    return (h->order == 5 || h->order == 6) && h->d.SKbf && h->d.tmapK_ok && h->N <= 64;
}

cudaError_t make_tck_tensor_map(hobo_instance* h)
{
    const auto& d = h->d;
    cudaError_t e = encode_planes_map(h->d.tmapK, d.SKbf, d.nsplitK, h->N, d.RK, 64, 256);
    h->d.tmapK_ok = e == cudaSuccess;
    return e;
}

cudaError_t launch_energy_tck(const hobo_instance* h, const uint32_t* X, int B, float* E, float* g_or_dE,
                              bool flip_out, cudaStream_t st)
{
    if (!tck_supported(h)) return cudaErrorNotSupported;
    if (B == 0) return cudaSuccess;
    const auto& d = h->d;
    cudaError_t e = cudaSuccess;
    if (h->low) {
        const int rc = energy_dispatch(h->low, X, B, E, g_or_dE, false, 0, st);
        if (rc != HOBO_OK) return cudaErrorUnknown;
    }
    const int tiles = (B + kTcM - 1) / kTcM;
    const int chunks = std::max(1, std::min(h->N, h->num_sms / tiles));
    TckParams p{};
    p.X = X; p.B = B; p.N = h->N; p.W = h->W; p.RK = d.RK; p.nsplit = d.nsplitK;
    p.T = tiles; p.chunks = chunks; p.G = tiles * chunks; p.status = h->status;
    p.rmask = d.kmask; p.rmin = d.kmin;
    float *Epart = nullptr, *GK = nullptr;
    e = cudaMallocAsync((void**)&Epart, sizeof(float) * (size_t)p.G * kTcM * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&GK, sizeof(float) * (size_t)B * h->N, st);
    p.Epart = Epart;
    p.GK = GK;
    const size_t sm = 1024 + 16384 + (size_t)kTcStages * 256 * 128 + 256;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(energy_tck_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) {
        const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(d.tmapK);
        energy_tck_kernel<<<p.G, kTcThreads, sm, st>>>(*map, p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        energy_tck_finalize<<<B, 64, 0, st>>>(Epart, GK, X, B, h->N, h->W, tiles, chunks, h->low ? 1 : 0,
                                              flip_out ? 1 : 0, E, g_or_dE);
        e = cudaGetLastError();
    }
    if (Epart) cudaFreeAsync(Epart, st);
    if (GK) cudaFreeAsync(GK, st);
    return e;
}

// ---------------------------------------------------------------------------
// Exact re-score on the tensor cores.  The fixed-point cubic coefficients
// C[m][j][l] (m < j < l) are split into rs_L signed 8-bit limbs, one bf16
// plane each (exact), and for a tile of 128 states each item (m, q) forms
// D_q[b][j] = sum_l limb_q[m][j][l] x_bl on the tensor cores.  Every term is
// an integer of magnitude <= 255 and K <= 256, so D_q is an exact integer
// below 2^24 in float32, and so is s_q = sum_j x_bj D_q[b][j] (at most 256
// such terms in four partial sums).  The epilogue adds x_bm * s_q * 2^(8q)
// to a 64-bit accumulator: the cubic energy sum_{m<j<l} C x_m x_j x_l
// exactly, the same integer as the CUDA-core re-score.  K blocks and
// accumulator columns that hold only zeros (l <= m + 1, j <= m) are
// skipped; items with no K block left are skipped by all three roles.
// ---------------------------------------------------------------------------
constexpr int kMaxChunks = 256;

struct TcExactParams {
    const uint32_t* X;
    int B, N, W, NJ, KP, L;
    int T, chunks, G;
    unsigned long long* acc;
    int* status;
    int mb[kMaxChunks + 1];   // m-chunk c is [mb[c], mb[c+1]), balanced by work
};

__global__ void __launch_bounds__(kTcThreads, 1)
energy_tc_exact_kernel(const __grid_constant__ CUtensorMap tmap, const TcExactParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int nKB = p.KP / kTcKB;
    const uint32_t stage_bytes = (uint32_t)p.NJ * 128u;
    uint8_t* sA = smem;
    uint8_t* sB = sA + nKB * 16384;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kTcStages * stage_bytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + kTcStages;
    uint64_t* afull = bars + 2 * kTcStages;
    uint64_t* aempty = afull + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(aempty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    volatile int* never_set = abort_flag + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = p.N, W = p.W, B = p.B;
    const int c = blockIdx.x;
    const int tile_c = c % p.T, chunk = c / p.T;
    const int i0 = tile_c * N + p.mb[chunk];
    const int i1 = tile_c * N + p.mb[chunk + 1];

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&afull[s], 1);
            mbar_init(&aempty[s], 4);
        }
        *abort_flag = 0;
        *never_set = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    int pstage = 0;
    uint32_t pphase = 0;
    uint32_t armed_phase[kTcStages];
    bool armed[kTcStages];
    for (int s = 0; s < kTcStages; ++s) { armed[s] = false; armed_phase[s] = 0; }
    int cstage = 0;
    uint32_t cphase = 0;
    int acc_mma = 0, acc_epi = 0;
    const uint32_t idesc = idesc_bf16(kTcM, p.NJ);

    for (int it = i0; it < i1;) {
        const int tile = it / N;
        const int seg_end = min(i1, (tile + 1) * N);
        {
            const int cpr = p.KP / 8;
            for (int q = threadIdx.x; q < kTcM * cpr; q += blockDim.x) {
                const int r = q / cpr, cc = q % cpr;
                const int kb = cc >> 3, ch = cc & 7;
                const int b = tile * kTcM + r;
                const int l0 = cc * 8;
                uint32_t byte = 0;
                if (b < B && l0 < N) {
                    byte = (p.X[(int64_t)b * W + (l0 >> 5)] >> (l0 & 31)) & 0xFFu;
                    const int rem = N - l0;
                    if (rem < 8) byte &= (1u << rem) - 1u;
                }
                uint32_t wv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t lo = ((byte >> (2 * e)) & 1u) ? 0x3F80u : 0u;
                    const uint32_t hi = ((byte >> (2 * e + 1)) & 1u) ? 0x3F80u : 0u;
                    wv[e] = lo | (hi << 16);
                }
                uint8_t* dst = sA + kb * 16384 + (r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4);
                *reinterpret_cast<uint4*>(dst) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();

        if (warp == 0) {
            if (lane == 0) {
                for (int j = it; j < seg_end && !*abort_flag; ++j) {
                    const int m = j % N;
                    const int kb0 = (m + 2) / kTcKB;     // l >= m + 2 only
                    if (kb0 >= nKB) continue;
                    for (int q = 0; q < p.L; ++q)
                        for (int kb = kb0; kb < nKB; ++kb) {
                            if (!mbar_wait(&empty[pstage], pphase ^ 1u, abort_flag)) {
                                set_abort(abort_flag, p.status);
                                break;
                            }
                            mbar_expect_tx(&full[pstage], stage_bytes);
                            tma_load_2d(sB + pstage * stage_bytes, &tmap, kb * kTcKB, (q * N + m) * p.NJ,
                                        &full[pstage]);
                            armed[pstage] = true;
                            armed_phase[pstage] = pphase;
                            if (++pstage == kTcStages) { pstage = 0; pphase ^= 1u; }
                        }
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {
                bool ok = true;
                for (int j = it; j < seg_end && ok && !*abort_flag; ++j) {
                    const int m = j % N;
                    const int kb0 = (m + 2) / kTcKB;
                    if (kb0 >= nKB) continue;
                    for (int q = 0; q < p.L && ok; ++q) {
                        const int buf = acc_mma & 1;
                        if (!mbar_wait(&aempty[buf], (((uint32_t)acc_mma >> 1) & 1u) ^ 1u, abort_flag)) {
                            set_abort(abort_flag, p.status);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d = tmem + (uint32_t)(buf * 256);
                        uint32_t accum = 0;
                        for (int kb = kb0; kb < nKB; ++kb) {
                            if (!mbar_wait(&full[cstage], cphase, abort_flag)) {
                                set_abort(abort_flag, p.status);
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint64_t ad = sw128_desc(smem_u32(sA + kb * 16384));
                            const uint64_t bd = sw128_desc(smem_u32(sB + cstage * stage_bytes));
#pragma unroll
                            for (int k = 0; k < kTcKB / 16; ++k) {
                                tc_mma(d, ad + 2 * k, bd + 2 * k, idesc, accum);
                                accum = 1;
                            }
                            tc_commit(&empty[cstage]);
                            if (++cstage == kTcStages) { cstage = 0; cphase ^= 1u; }
                        }
                        if (!ok) break;
                        tc_commit(&afull[buf]);
                        ++acc_mma;
                    }
                }
            }
        } else {
            const int quad = warp & 3;
            const int r = quad * 32 + lane;
            const int b = tile * kTcM + r;
            uint32_t x[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                uint32_t v = (b < B && k < W) ? p.X[(int64_t)b * W + k] : 0u;
                const int rem = N - 32 * k;
                if (rem <= 0) v = 0u; else if (rem < 32) v &= (1u << rem) - 1u;
                x[k] = v;
            }
            long long e3 = 0;
            const int nch = (p.NJ + 31) / 32;
            bool ok = true;
            for (int j = it; j < seg_end && ok; ++j) {
                const int m = j % N;
                const int kb0 = (m + 2) / kTcKB;
                if (kb0 >= nKB) continue;
                uint32_t xmw = x[0];
#pragma unroll
                for (int k = 1; k < 8; ++k) xmw = ((m >> 5) == k) ? x[k] : xmw;
                const bool xm = (xmw >> (m & 31)) & 1u;
                const int ch0 = (m + 1) >> 5;             // columns j <= m hold zeros
                for (int q = 0; q < p.L; ++q) {
                    const int buf = acc_epi & 1;
                    ok = __all_sync(0xffffffffu, mbar_wait(&afull[buf], ((uint32_t)acc_epi >> 1) & 1u, abort_flag));
                    if (!ok) {
                        if (lane == 0) set_abort(abort_flag, p.status);
                        break;
                    }
                    tc_fence_after();
                    float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
                    const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 256);
#pragma unroll 1
                    for (int ch = ch0; ch < nch; ++ch) {
                        uint32_t v[32];
                        tmem_ld32(tbase + (uint32_t)(ch * 32), v);
                        tmem_ld_wait();
                        uint32_t xw = x[0];
#pragma unroll
                        for (int k = 1; k < 8; ++k) xw = (ch == k) ? x[k] : xw;
#pragma unroll
                        for (int t = 0; t < 32; t += 4) {
                            if ((xw >> t) & 1u) c0 = __fadd_rn(c0, __uint_as_float(v[t]));
                            if ((xw >> (t + 1)) & 1u) c1 = __fadd_rn(c1, __uint_as_float(v[t + 1]));
                            if ((xw >> (t + 2)) & 1u) c2 = __fadd_rn(c2, __uint_as_float(v[t + 2]));
                            if ((xw >> (t + 3)) & 1u) c3 = __fadd_rn(c3, __uint_as_float(v[t + 3]));
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&aempty[buf]);
                    ++acc_epi;
                    if (xm) {
                        const long long sq = __float2ll_rn(__fadd_rn(__fadd_rn(c0, c1), __fadd_rn(c2, c3)));
                        e3 += sq * (1LL << (8 * q));
                    }
                }
            }
            if (b < B && e3 != 0) atomicAdd(p.acc + b, (unsigned long long)e3);
        }
        __syncthreads();
        it = seg_end;
    }

    if (warp == 0 && lane == 0 && *abort_flag) {
        for (int s = 0; s < kTcStages; ++s)
            if (armed[s]) (void)mbar_wait(&full[s], armed_phase[s], never_set);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// Exact linear and pair parts: acc[b] += sum_m x_bm (a[m] + sum_{j>m} x_bj S2[m][j])
// in 64-bit fixed point.  A block takes 128 states and a chunk of rows m.
__global__ void __launch_bounds__(kPairThreads)
pair_exact_kernel(const uint32_t* __restrict__ X, int B, int N, int W, const long long* __restrict__ a,
                  const long long* __restrict__ S2, int mchunk, unsigned long long* __restrict__ acc)
{
    __shared__ long long row[256];
    const int b = blockIdx.x * kPairThreads + threadIdx.x;
    uint32_t x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        uint32_t v = (b < B && k < W) ? X[(int64_t)b * W + k] : 0u;
        const int rem = N - 32 * k;
        if (rem <= 0) v = 0u; else if (rem < 32) v &= (1u << rem) - 1u;
        x[k] = v;
    }
    long long s = 0;
    const int m0 = blockIdx.y * mchunk, m1 = min(N, m0 + mchunk);
    for (int m = m0; m < m1; ++m) {
        __syncthreads();
        for (int j = threadIdx.x; j < N; j += kPairThreads) row[j] = __ldg(S2 + (int64_t)m * N + j);
        __syncthreads();
        uint32_t xmw = x[0];
#pragma unroll
        for (int k = 1; k < 8; ++k) xmw = ((m >> 5) == k) ? x[k] : xmw;
        if (!((xmw >> (m & 31)) & 1u)) continue;
        long long t = __ldg(a + m);
#pragma unroll 1
        for (int k = (m + 1) >> 5; k < W; ++k) {
            uint32_t xw = x[0];
#pragma unroll
            for (int k2 = 1; k2 < 8; ++k2) xw = (k == k2) ? x[k2] : xw;
            if (32 * k <= m) xw &= ~((2u << (m & 31)) - 1u);   // j > m only
#pragma unroll 4
            for (int u = 0; u < 32; ++u)
                if ((xw >> u) & 1u) t += row[32 * k + u];
        }
        s += t;
    }
    if (b < B && s != 0) atomicAdd(acc + b, (unsigned long long)s);
}

bool exact_tc_supported(const hobo_instance* h)
{
    return h->dense && h->d.S3limb && h->d.tmap_rs_ok && h->N <= 256;
}

// acc (B zeroed words) += exact fixed-point energies (scale 2^rs_shift)
cudaError_t launch_energy_exact_tc(const hobo_instance* h, const uint32_t* X, int B, unsigned long long* acc,
                                   cudaStream_t st)
{
    if (!exact_tc_supported(h)) return cudaErrorNotSupported;
    if (B == 0) return cudaSuccess;
    const auto& d = h->d;
    {
        const int btiles = (B + kPairThreads - 1) / kPairThreads;
        const int mch = std::max(1, std::min(h->N, (2 * h->num_sms + btiles - 1) / btiles));
        const int mchunk = (h->N + mch - 1) / mch;
        pair_exact_kernel<<<dim3(btiles, (h->N + mchunk - 1) / mchunk), kPairThreads, 0, st>>>(
            X, B, h->N, h->W, d.rs_a, d.rs_S2, mchunk, acc);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int tiles = (B + kTcM - 1) / kTcM;
    const int chunks = std::max(1, std::min(std::min(h->N, kMaxChunks), h->num_sms / tiles));
    TcExactParams p{};
    p.X = X; p.B = B; p.N = h->N; p.W = h->W; p.NJ = d.NJ; p.KP = d.KP; p.L = d.rs_L;
    p.T = tiles; p.chunks = chunks; p.G = tiles * chunks; p.acc = acc; p.status = h->status;
    {
        // m-chunk boundaries at equal shares of the work: item m has
        // nKB - (m+2)/64 K blocks (none for the last m) plus its epilogue
        const int nKB = d.KP / kTcKB;
        std::vector<double> cum((size_t)h->N + 1, 0.0);
        for (int m = 0; m < h->N; ++m) cum[m + 1] = cum[m] + std::max(0, nKB - (m + 2) / kTcKB) + 0.25;
        p.mb[0] = 0;
        int m = 0;
        for (int k = 1; k < chunks; ++k) {
            const double want = cum[h->N] * k / chunks;
            while (m < h->N && cum[m + 1] <= want) ++m;
            p.mb[k] = std::max(p.mb[k - 1], m);
        }
        p.mb[chunks] = h->N;
    }
    const size_t sm = tc_smem_bytes(d.NJ, d.KP);
    cudaError_t e = cudaFuncSetAttribute(energy_tc_exact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(d.tmap_rs);
    energy_tc_exact_kernel<<<p.G, kTcThreads, sm, st>>>(*map, p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact energies and fields on the tensor cores.  The fixed-point
// coefficients C = round(c * 2^S) of every monomial containing m sit in m's
// slab: a cubic {m, j, l} at row j, column l > j (the upper triangle), a
// pair {m, j} on the diagonal (j, j); each plane holds one 8-bit limb of
// them (exact bf16).  For a tile of 128 states and an item (m, limb q) the
// tensor cores form
//   D_q[b][j] = sum_{l >= j} limb_q[m][j][l] x_bl
// whose products are integers of magnitude <= 255 and whose sums stay below
// 2^24, so they are exact in float32, and so are the epilogue's sums over
// the set bits j of the state below and above m,
//   u_q = sum_{j < m} x_bj D_q[b][j],   t_q = sum_{j > m} x_bj D_q[b][j].
// With t = sum_q t_q 2^(8q) and s = t + sum_q u_q 2^(8q) (64-bit integers):
//   g_bm = a_m + s   (the field: every pair and cubic term containing m),
//   E_b  = sum_m x_bm (a_m + t)   (t: the terms whose smallest member is m),
// each rounded once to float32 -- the term-list path's values, bit for bit.
// Only the triangle is fed to the tensor cores: K block kb (l in
// [64 kb, 64 kb + 64)) meets rows j < 64 (kb + 1), so its MMAs run with
// N = 64 (kb + 1) columns, largest first (that one clears the accumulator):
// 10/16 of the full slab for N = 256.
// ---------------------------------------------------------------------------
struct TcFixParams {
    const uint32_t* X;
    int B, N, W, KP, L, S;
    int T, chunks, G;
    const long long* fa;     // [N]
    float* out_g;
    int flip;
    unsigned long long* Epart;   // [G][128]: this chunk's part of the fixed-point energy (mod 2^64)
    int* status;
};

// Adds the accumulator columns whose bit is set in xw into four partial
// sums (exact: integers below 2^24).
__device__ __forceinline__ void add_set_columns(const uint32_t (&v)[32], uint32_t xw, float (&c)[4])
{
#pragma unroll
    for (int t = 0; t < 32; t += 4) {
        if ((xw >> t) & 1u) c[0] = __fadd_rn(c[0], __uint_as_float(v[t]));
        if ((xw >> (t + 1)) & 1u) c[1] = __fadd_rn(c[1], __uint_as_float(v[t + 1]));
        if ((xw >> (t + 2)) & 1u) c[2] = __fadd_rn(c[2], __uint_as_float(v[t + 2]));
        if ((xw >> (t + 3)) & 1u) c[3] = __fadd_rn(c[3], __uint_as_float(v[t + 3]));
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
energy_tc_fix_kernel(const __grid_constant__ CUtensorMap tmap, const TcFixParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int nKB = p.KP / kTcKB;
    const uint32_t stage_bytes = (uint32_t)p.KP * 128u;
    uint8_t* sA = smem;
    uint8_t* sB = sA + nKB * 16384;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kTcStages * stage_bytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + kTcStages;
    uint64_t* afull = bars + 2 * kTcStages;
    uint64_t* aempty = afull + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(aempty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    volatile int* never_set = abort_flag + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = p.N, W = p.W, B = p.B;
    const int c = blockIdx.x;
    const int tile_c = c % p.T, chunk = c / p.T;
    const int i0 = tile_c * N + (int)((int64_t)chunk * N / p.chunks);
    const int i1 = tile_c * N + (int)((int64_t)(chunk + 1) * N / p.chunks);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&afull[s], 1);
            mbar_init(&aempty[s], 4);
        }
        *abort_flag = 0;
        *never_set = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    int pstage = 0;
    uint32_t pphase = 0;
    uint32_t armed_phase[kTcStages];
    bool armed[kTcStages];
    for (int s = 0; s < kTcStages; ++s) { armed[s] = false; armed_phase[s] = 0; }
    int cstage = 0;
    uint32_t cphase = 0;
    int acc_mma = 0, acc_epi = 0;

    for (int it = i0; it < i1;) {
        const int tile = it / N;
        const int seg_end = min(i1, (tile + 1) * N);
        {
            const int cpr = p.KP / 8;
            for (int q = threadIdx.x; q < kTcM * cpr; q += blockDim.x) {
                const int r = q / cpr, cc = q % cpr;
                const int kb = cc >> 3, ch = cc & 7;
                const int b = tile * kTcM + r;
                const int l0 = cc * 8;
                uint32_t byte = 0;
                if (b < B && l0 < N) {
                    byte = (p.X[(int64_t)b * W + (l0 >> 5)] >> (l0 & 31)) & 0xFFu;
                    const int rem = N - l0;
                    if (rem < 8) byte &= (1u << rem) - 1u;
                }
                uint32_t wv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t lo = ((byte >> (2 * e)) & 1u) ? 0x3F80u : 0u;
                    const uint32_t hi = ((byte >> (2 * e + 1)) & 1u) ? 0x3F80u : 0u;
                    wv[e] = lo | (hi << 16);
                }
                uint8_t* dst = sA + kb * 16384 + (r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4);
                *reinterpret_cast<uint4*>(dst) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();

        if (warp == 0) {
            if (lane == 0) {
                // ---- producer: rows j < 64 (kb + 1) of K block kb, kb descending
                bool ok = true;
                for (int j = it; j < seg_end && ok && !*abort_flag; ++j) {
                    const int m = j % N;
                    for (int q = 0; q < p.L && ok; ++q)
                        for (int kb = nKB - 1; kb >= 0; --kb) {
                            if (!mbar_wait(&empty[pstage], pphase ^ 1u, abort_flag)) {
                                set_abort(abort_flag, p.status);
                                ok = false;
                                break;
                            }
                            mbar_expect_tx(&full[pstage], (uint32_t)(kb + 1) * 64u * 128u);
                            for (int rb = 0; rb <= kb; ++rb)
                                tma_load_2d(sB + pstage * stage_bytes + rb * 8192, &tmap, kb * kTcKB,
                                            (q * N + m) * p.KP + rb * 64, &full[pstage]);
                            armed[pstage] = true;
                            armed_phase[pstage] = pphase;
                            if (++pstage == kTcStages) { pstage = 0; pphase ^= 1u; }
                        }
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {
                // ---- MMA issuer: one accumulator per item (m, q)
                bool ok = true;
                for (int j = it; j < seg_end && ok && !*abort_flag; ++j) {
                    for (int q = 0; q < p.L && ok; ++q) {
                        const int buf = acc_mma & 1;
                        if (!mbar_wait(&aempty[buf], (((uint32_t)acc_mma >> 1) & 1u) ^ 1u, abort_flag)) {
                            set_abort(abort_flag, p.status);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d = tmem + (uint32_t)(buf * 256);
                        uint32_t accum = 0;
                        for (int kb = nKB - 1; kb >= 0; --kb) {
                            if (!mbar_wait(&full[cstage], cphase, abort_flag)) {
                                set_abort(abort_flag, p.status);
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t idesc = idesc_bf16(kTcM, 64 * (kb + 1));
                            const uint64_t ad = sw128_desc(smem_u32(sA + kb * 16384));
                            const uint64_t bd = sw128_desc(smem_u32(sB + cstage * stage_bytes));
#pragma unroll
                            for (int k = 0; k < kTcKB / 16; ++k) {
                                tc_mma(d, ad + 2 * k, bd + 2 * k, idesc, accum);
                                accum = 1;
                            }
                            tc_commit(&empty[cstage]);
                            if (++cstage == kTcStages) { cstage = 0; cphase ^= 1u; }
                        }
                        if (!ok) break;
                        tc_commit(&afull[buf]);
                        ++acc_mma;
                    }
                }
            }
        } else {
            // ---- epilogue: thread = TMEM lane = state row
            const int quad = warp & 3;
            const int r = quad * 32 + lane;
            const int b = tile * kTcM + r;
            uint32_t x[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                uint32_t v = (b < B && k < W) ? p.X[(int64_t)b * W + k] : 0u;
                const int rem = N - 32 * k;
                if (rem <= 0) v = 0u; else if (rem < 32) v &= (1u << rem) - 1u;
                x[k] = v;
            }
            unsigned long long esum = 0;
            const int nch = (N + 31) / 32;
            bool ok = true;
            for (int j = it; j < seg_end && ok; ++j) {
                const int m = j % N;
                const int mch = m >> 5;
                // bits of the chunk holding m: above m / below m
                const uint32_t above_m = (m & 31) == 31 ? 0u : (0xFFFFFFFFu << ((m & 31) + 1));
                unsigned long long sf = 0, tf = 0;
                for (int q = 0; q < p.L; ++q) {
                    const int buf = acc_epi & 1;
                    ok = __all_sync(0xffffffffu, mbar_wait(&afull[buf], ((uint32_t)acc_epi >> 1) & 1u, abort_flag));
                    if (!ok) {
                        if (lane == 0) set_abort(abort_flag, p.status);
                        break;
                    }
                    tc_fence_after();
                    float lo[4] = {0.f, 0.f, 0.f, 0.f}, hi[4] = {0.f, 0.f, 0.f, 0.f};
                    const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 256);
#pragma unroll 1
                    for (int ch = 0; ch < nch; ++ch) {
                        uint32_t v[32];
                        tmem_ld32(tbase + (uint32_t)(ch * 32), v);
                        tmem_ld_wait();
                        uint32_t xw = x[0];
#pragma unroll
                        for (int k = 1; k < 8; ++k) xw = (ch == k) ? x[k] : xw;
                        if (ch < mch) {
                            add_set_columns(v, xw, lo);
                        } else if (ch > mch) {
                            add_set_columns(v, xw, hi);
                        } else {
                            add_set_columns(v, xw & ~above_m, lo);
                            add_set_columns(v, xw & above_m, hi);
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&aempty[buf]);
                    ++acc_epi;
                    const long long uq = __float2ll_rn(__fadd_rn(__fadd_rn(lo[0], lo[1]), __fadd_rn(lo[2], lo[3])));
                    const long long tq = __float2ll_rn(__fadd_rn(__fadd_rn(hi[0], hi[1]), __fadd_rn(hi[2], hi[3])));
                    tf += (unsigned long long)tq << (8 * q);
                    sf += (unsigned long long)(uq + tq) << (8 * q);
                }
                if (!ok) break;
                const unsigned long long am = (unsigned long long)__ldg(p.fa + m);
                uint32_t xmw = x[0];
#pragma unroll
                for (int k = 1; k < 8; ++k) xmw = (mch == k) ? x[k] : xmw;
                const bool xm = (xmw >> (m & 31)) & 1u;
                if (xm) esum += am + tf;
                if (b < B && p.out_g) {
                    const float g = scalbnf(__ll2float_rn((long long)(am + sf)), -p.S);
                    p.out_g[(int64_t)b * N + m] = (p.flip && xm) ? -g : g;
                }
            }
            p.Epart[(int64_t)c * kTcM + r] = esum;
        }
        __syncthreads();
        it = seg_end;
    }

    if (warp == 0 && lane == 0 && *abort_flag) {
        for (int s = 0; s < kTcStages; ++s)
            if (armed[s]) (void)mbar_wait(&full[s], armed_phase[s], never_set);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// E_b: the fixed-point parts of the m-chunks of its tile, added (modulo
// 2^64; the total fits in 63 bits) and rounded once to float32.
__global__ void energy_tc_fix_finalize(const unsigned long long* __restrict__ Epart, int B, int T, int chunks,
                                       int S, float* __restrict__ E)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int t = b / kTcM, r = b % kTcM;
    unsigned long long s = 0;
    for (int k = 0; k < chunks; ++k) s += Epart[(int64_t)(k * T + t) * kTcM + r];
    E[b] = scalbnf(__ll2float_rn((long long)s), -S);
}

bool fix_tc_supported(const hobo_instance* h)
{
    return h->dense && h->d.S3flimb && h->d.tmap_fl_ok && h->N <= 256;
}

cudaError_t make_tc_tensor_map_fl(hobo_instance* h)
{
    const auto& d = h->d;
    cudaError_t e = encode_planes_map(h->d.tmap_fl, d.S3flimb, d.fl_L, h->N, d.KP, d.KP, 64);
    h->d.tmap_fl_ok = e == cudaSuccess;
    return e;
}

cudaError_t launch_energy_tc_fix(const hobo_instance* h, const uint32_t* X, int B, float* E, float* g_or_dE,
                                 bool flip_out, cudaStream_t st)
{
    if (!fix_tc_supported(h)) return cudaErrorNotSupported;
    if (B == 0) return cudaSuccess;
    const auto& d = h->d;
    const int tiles = (B + kTcM - 1) / kTcM;
    const int chunks = std::max(1, std::min(h->N, h->num_sms / tiles));
    TcFixParams p{};
    p.X = X; p.B = B; p.N = h->N; p.W = h->W; p.KP = d.KP; p.L = d.fl_L; p.S = d.fl_shift;
    p.T = tiles; p.chunks = chunks; p.G = tiles * chunks;
    p.fa = d.fa; p.out_g = g_or_dE; p.flip = flip_out ? 1 : 0; p.status = h->status;
    unsigned long long* Epart = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&Epart, sizeof(unsigned long long) * (size_t)p.G * kTcM, st);
    if (e != cudaSuccess) return e;
    p.Epart = Epart;
    const size_t sm = tc_smem_bytes(d.KP, d.KP);
    e = cudaFuncSetAttribute(energy_tc_fix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) {
        const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(d.tmap_fl);
        energy_tc_fix_kernel<<<p.G, kTcThreads, sm, st>>>(*map, p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        energy_tc_fix_finalize<<<(B + 255) / 256, 256, 0, st>>>(Epart, B, tiles, chunks, p.S, E);
        e = cudaGetLastError();
    }
    cudaFreeAsync(Epart, st);
    return e;
}

cudaError_t launch_energy_tc(const hobo_instance* h, const uint32_t* X, int B, float* E, float* g_or_dE,
                             bool flip_out, cudaStream_t st)
{
    if (!tc_supported(h)) return cudaErrorNotSupported;
    if (B == 0) return cudaSuccess;
    const auto& d = h->d;
    const int tiles = (B + kTcM - 1) / kTcM;
    const int chunks = std::max(1, std::min(h->N, h->num_sms / tiles));
    const int G = tiles * chunks;
    TcParams p{};
    p.X = X; p.B = B; p.N = h->N; p.W = h->W; p.NJ = d.NJ; p.KP = d.KP; p.nsplit = d.nsplit;
    p.P = (h->N + 3) & ~3; p.a = d.a; p.out_g = g_or_dE; p.flip = flip_out ? 1 : 0;
    p.T = tiles; p.chunks = chunks; p.G = G; p.status = h->status;
    float* Epart = nullptr;
    float* Qt = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&Epart, sizeof(float) * (size_t)G * kTcM * 4, st);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync((void**)&Qt, sizeof(float) * (size_t)h->N * B, st);
    if (e != cudaSuccess) { cudaFreeAsync(Epart, st); return e; }
    p.Epart = Epart;
    p.Qt = Qt;
    {
        const int btiles = (B + kPairThreads - 1) / kPairThreads;
        const int mch = std::max(1, std::min(h->N, (2 * h->num_sms + btiles - 1) / btiles));
        const int mchunk = (h->N + mch - 1) / mch;
        pair_fields_kernel<<<dim3(btiles, (h->N + mchunk - 1) / mchunk), kPairThreads, 0, st>>>(
            X, B, h->N, h->W, d.S2, p.P, mchunk, Qt);
        e = cudaGetLastError();
    }
    const size_t sm = tc_smem_bytes(d.NJ, d.KP);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(energy_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) {
        const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(d.tmap);
        energy_tc_kernel<<<G, kTcThreads, sm, st>>>(*map, p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        energy_tc_finalize<<<(B + 255) / 256, 256, 0, st>>>(Epart, B, tiles, chunks, E);
        e = cudaGetLastError();
    }
    cudaFreeAsync(Epart, st);
    cudaFreeAsync(Qt, st);
    return e;
}

}  // namespace hobo
