// CUDA-core kernels: random initial states, term-list energy/field
// contraction (float32), float64 re-scoring, and the Metropolis sweeps
// (tuned warp-per-state kernel and the plain thread-per-state kernel).
#include <algorithm>
#include <type_traits>
#include "hobo_internal.h"
#include "hobo_dev.cuh"
#include "sweep_impl.cuh"

namespace hobo {

// ===========================================================================
// Initial states: bit i of state b is bit 31 of word (i % 4) of
// Philox(counter = (i/4, 0, b, 1), key = seed).
// ===========================================================================
__global__ void init_states_kernel(uint32_t* __restrict__ X, int B, int N, int W,
                                   uint32_t k0, uint32_t k1)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)B * W) return;
    const int b = (int)(tid / W), w = (int)(tid % W);
    X[tid] = init_word(b, w, N, k0, k1);
}

cudaError_t launch_init_states(uint32_t* X, int B, int N, int W, uint64_t seed, cudaStream_t st)
{
    if (B == 0) return cudaSuccess;
    const int64_t n = (int64_t)B * W;
    const int threads = 256;
    init_states_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
        X, B, N, W, (uint32_t)seed, (uint32_t)(seed >> 32));
    return cudaGetLastError();
}

// ===========================================================================
// Term-list contraction on CUDA cores.  A block holds 32 states (one per
// lane) with their bits transposed in shared memory (word w of state b at
// [w][b], plus the sentinel bit N that reads as 1).  Warps split the
// variables: for variable j the field is the sum of the coefficients of the
// monomials containing j whose other members are all set.  The energy is
// the sum over monomials whose members are all set.
// ===========================================================================
constexpr int kTermThreads = 256;

// Compensated summation (Kahan): acc + comp tracks the exact running sum to
// within a few units in the last place, whatever the number of terms.
__device__ __forceinline__ void kahan_add(float& acc, float& comp, float v)
{
    const float y = __fsub_rn(v, comp);
    const float t = __fadd_rn(acc, y);
    comp = __fsub_rn(__fsub_rn(t, acc), y);
    acc = t;
}

template <bool FLIP>
__global__ void __launch_bounds__(kTermThreads)
energy_terms_kernel(const uint32_t* __restrict__ X, int B, int N, int W,
                    const int64_t* __restrict__ fptr, const uint16_t* __restrict__ fvars,
                    const float* __restrict__ fcoef, int KF,
                    const uint16_t* __restrict__ tvars, const float* __restrict__ tcoef,
                    int64_t M, int K, int KS, float* __restrict__ out_g, float* __restrict__ out_E)
{
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int b0 = blockIdx.x * 32;
    const int nb = min(32, B - b0);
    const int WS = W + 1;
    uint32_t* bits = smem;                              // [WS][32]
    float* red = reinterpret_cast<float*>(bits + WS * 32);   // [nwarps][32]
    float* gs = red + nwarps * 32;                      // [32][N+1]
    const int NP = N + 1;

    for (int q = threadIdx.x; q < WS * 32; q += blockDim.x) {
        const int w = q >> 5, b = q & 31;
        uint32_t v = 0;
        if (w < W && b < nb) {
            v = X[(int64_t)(b0 + b) * W + w];
            const int rem = N - 32 * w;
            if (rem < 32) v &= (1u << rem) - 1u;
        }
        if (w == (N >> 5)) v |= 1u << (N & 31);
        bits[q] = v;
    }
    __syncthreads();

    if (out_g) {
        for (int j = warp; j < N; j += nwarps) {
            float acc = 0.0f, comp = 0.0f;   // compensated (Kahan) sum
            const int64_t e1 = fptr[j + 1];
            for (int64_t e = fptr[j]; e < e1; ++e) {
                const float c = fcoef[e];
                uint32_t p = 1u;
                for (int s = 0; s < KF; ++s) {
                    const int v = fvars[e * KF + s];
                    p &= bits[(v >> 5) * 32 + lane] >> (v & 31);
                }
                if (p & 1u) kahan_add(acc, comp, c);
            }
            if (FLIP && ((bits[(j >> 5) * 32 + lane] >> (j & 31)) & 1u)) acc = -acc;
            gs[lane * NP + j] = acc;
        }
    }

    float eacc = 0.0f, ecomp = 0.0f;
    for (int64_t t = warp; t < M; t += nwarps) {
        const float c = tcoef[t];
        uint32_t p = 1u;
        for (int s = 0; s < K; ++s) {
            const int v = tvars[t * KS + s];
            p &= bits[(v >> 5) * 32 + lane] >> (v & 31);
        }
        if (p & 1u) kahan_add(eacc, ecomp, c);
    }
    red[warp * 32 + lane] = eacc;
    __syncthreads();
    if (warp == 0 && lane < nb) {
        float e = 0.0f;
        for (int q = 0; q < nwarps; ++q) e = __fadd_rn(e, red[q * 32 + lane]);
        out_E[b0 + lane] = e;
    }
    if (out_g) {
        for (int b = 0; b < nb; ++b)
            for (int j = threadIdx.x; j < N; j += blockDim.x)
                out_g[(int64_t)(b0 + b) * N + j] = gs[b * NP + j];
    }
}

static size_t term_smem(int N, int W, bool with_g)
{
    return sizeof(uint32_t) * (size_t)(W + 1) * 32 + sizeof(float) * (kTermThreads / 32) * 32 +
           (with_g ? sizeof(float) * 32 * (size_t)(N + 1) : 0);
}

cudaError_t launch_energy_terms(const hobo_instance* h, const uint32_t* X, int B, float* E,
                                float* g_or_dE, bool flip_out, cudaStream_t st)
{
    if (B == 0) return cudaSuccess;
    const size_t sm = term_smem(h->N, h->W, g_or_dE != nullptr);
    const unsigned grid = (unsigned)((B + 31) / 32);
    const auto& d = h->d;
    if (flip_out) {
        cudaFuncSetAttribute(energy_terms_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        energy_terms_kernel<true><<<grid, kTermThreads, sm, st>>>(
            X, B, h->N, h->W, d.fptr, d.fvars, d.fcoef, h->KF, d.tvars, d.tcoef32, d.M, h->order, h->KS,
            g_or_dE, E);
    } else {
        cudaFuncSetAttribute(energy_terms_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        energy_terms_kernel<false><<<grid, kTermThreads, sm, st>>>(
            X, B, h->N, h->W, d.fptr, d.fvars, d.fcoef, h->KF, d.tvars, d.tcoef32, d.M, h->order, h->KS,
            g_or_dE, E);
    }
    return cudaGetLastError();
}

// ===========================================================================
// float64 re-scoring.  Each folded coefficient is held as the 64-bit integer
// round(c * 2^S), with S chosen per instance so that the sum of all
// |coefficients| stays below 2^62; the energy of a state is the exact
// integer sum of the coefficients of its active monomials, scaled by 2^-S
// and rounded once to float64.  Integer instances are exact; otherwise the
// error is at most (number of terms) * 2^-(S+1), below the rounding error of
// a float64 summation of the same terms.  Blocks take 32 states (one per
// lane) and a slice of the monomial list; slices are combined with 64-bit
// integer atomics, whose result does not depend on their order.
// ===========================================================================
constexpr int kFixThreads = 256;

template <int KS>
__global__ void __launch_bounds__(kFixThreads)
energy_fix_kernel(const uint32_t* __restrict__ X, int B, int N, int W,
                  const uint16_t* __restrict__ tvars, const long long* __restrict__ tfix,
                  int64_t M, int64_t per_slice, unsigned long long* __restrict__ acc)
{
    using Row = typename std::conditional<KS == 4, uint2, uint4>::type;   // KS u16 slots
    constexpr int U = 4;   // monomials in flight per warp
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int b0 = blockIdx.x * 32;
    const int nb = min(32, B - b0);
    const int WS = W + 1;
    uint32_t* bits = smem;
    long long* red = reinterpret_cast<long long*>(bits + ((WS * 32 + 1) & ~1));
    for (int q = threadIdx.x; q < WS * 32; q += blockDim.x) {
        const int w = q >> 5, b = q & 31;
        uint32_t v = 0;
        if (w < W && b < nb) {
            v = X[(int64_t)(b0 + b) * W + w];
            const int rem = N - 32 * w;
            if (rem < 32) v &= (1u << rem) - 1u;
        }
        if (w == (N >> 5)) v |= 1u << (N & 31);
        bits[q] = v;
    }
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.y * per_slice;
    const int64_t t1 = min(M, t0 + per_slice);
    const Row* rows = reinterpret_cast<const Row*>(tvars);
    long long s = 0;
    for (int64_t t = t0 + (int64_t)warp * U; t < t1; t += (int64_t)nwarps * U) {
        Row r[U];
        long long c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = t + u < t1;
            r[u] = ok ? __ldg(rows + t + u) : Row{};
            c[u] = ok ? __ldg(tfix + t + u) : 0ll;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t* wv = reinterpret_cast<const uint32_t*>(&r[u]);
            uint32_t p = 1u;
#pragma unroll
            for (int q = 0; q < KS / 2; ++q) {
                const int v0 = wv[q] & 0xFFFFu, v1 = wv[q] >> 16;
                p &= bits[(v0 >> 5) * 32 + lane] >> (v0 & 31);
                p &= bits[(v1 >> 5) * 32 + lane] >> (v1 & 31);
            }
            if (p & 1u) s += c[u];
        }
    }
    red[warp * 32 + lane] = s;
    __syncthreads();
    if (warp == 0 && lane < nb) {
        long long tot = 0;
        for (int q = 0; q < nwarps; ++q) tot += red[q * 32 + lane];
        atomicAdd(acc + b0 + lane, (unsigned long long)tot);
    }
}

// Dense order-3 instances: the same exact fixed-point sums, structured by
// the dense layout.  Lanes are 32 states; warps take pairs (m, j), m < j.
// For a pair the quadratic coefficient is added where both bits are set, and
// the cubic row C[m][j][l], l > j, is loaded once per 32 columns and
// broadcast lane by lane, so every coefficient is read once per 32 states.
template <int WMAX>
__global__ void __launch_bounds__(kFixThreads)
energy_fix_dense_kernel(const uint32_t* __restrict__ X, int B, int N, int W,
                        const long long* __restrict__ C3, const long long* __restrict__ S2f,
                        const long long* __restrict__ af, const uint16_t* __restrict__ pm,
                        const uint16_t* __restrict__ pj, int npairs, int per_slice,
                        unsigned long long* __restrict__ acc)
{
    __shared__ long long red[kFixThreads];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int b = blockIdx.x * 32 + lane;
    uint32_t x[WMAX];
#pragma unroll
    for (int k = 0; k < WMAX; ++k) {
        uint32_t v = (b < B && k < W) ? X[(int64_t)b * W + k] : 0u;
        const int rem = N - 32 * k;
        if (rem <= 0) v = 0u; else if (rem < 32) v &= (1u << rem) - 1u;
        x[k] = v;
    }
    long long s = 0;
    if (blockIdx.y == 0 && warp == 0)
        for (int m = 0; m < N; ++m)
            if ((sel_word(x, m >> 5) >> (m & 31)) & 1u) s += __ldg(af + m);
    const int p0 = blockIdx.y * per_slice, p1 = min(npairs, p0 + per_slice);
    for (int q = p0 + warp; q < p1; q += nwarps) {
        const int m = pm[q], j = pj[q];
        const bool mj = ((sel_word(x, m >> 5) >> (m & 31)) & (sel_word(x, j >> 5) >> (j & 31)) & 1u) != 0u;
        if (!__any_sync(0xffffffffu, mj)) continue;
        if (mj) s += __ldg(S2f + (int64_t)m * N + j);
        const long long* row = C3 + ((int64_t)m * N + j) * N;
        for (int k = (j + 1) >> 5; k < W; ++k) {
            const int l = 32 * k + lane;
            const long long c = l < N ? __ldg(row + l) : 0ll;
            const uint32_t xw = mj ? sel_word(x, k) : 0u;   // no cubic term without x_m x_j
#pragma unroll
            for (int t = 0; t < 32; ++t) {
                const long long ct = __shfl_sync(0xffffffffu, c, t);
                if ((xw >> t) & 1u) s += ct;
            }
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    if (warp == 0 && b < B) {
        long long tot = 0;
        for (int q = 0; q < nwarps; ++q) tot += red[q * 32 + lane];
        atomicAdd(acc + b, (unsigned long long)tot);
    }
}

static cudaError_t launch_fix_dense(const hobo_instance* h, const uint32_t* X, int B,
                                    unsigned long long* acc, cudaStream_t st)
{
    const auto& d = h->d;
    const int tiles = (B + 31) / 32;
    const int npairs = h->N * (h->N - 1) / 2;
    const int slices = std::max(1, std::min((4 * h->num_sms + tiles - 1) / tiles, (npairs + 63) / 64));
    const int per = (npairs + slices - 1) / slices;
    const dim3 grid(tiles, slices);
    if (h->W <= 8)
        energy_fix_dense_kernel<8><<<grid, kFixThreads, 0, st>>>(X, B, h->N, h->W, d.C3fix, d.S2fix, d.afix,
                                                                 d.pair_m, d.pair_j, npairs, per, acc);
    else
        energy_fix_dense_kernel<16><<<grid, kFixThreads, 0, st>>>(X, B, h->N, h->W, d.C3fix, d.S2fix, d.afix,
                                                                  d.pair_m, d.pair_j, npairs, per, acc);
    return cudaGetLastError();
}

__global__ void energy_fix_finalize(const unsigned long long* __restrict__ acc, int B, int S,
                                    double* __restrict__ E)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) E[b] = ldexp((double)(long long)acc[b], -S);
}

cudaError_t launch_energy_fp64(const hobo_instance* h, const uint32_t* X, int B, double* E,
                               cudaStream_t st)
{
    if (B == 0) return cudaSuccess;
    const int64_t M = h->d.M;
    const int tiles = (B + 31) / 32;
    int slices = (int)std::max<int64_t>(1, std::min<int64_t>((4LL * h->num_sms + tiles - 1) / tiles,
                                                             (M + 4095) / 4096));
    const int64_t per = (M + slices - 1) / std::max(slices, 1);
    unsigned long long* acc = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&acc, sizeof(unsigned long long) * (size_t)B, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (size_t)B, st);
    if (e == cudaSuccess && h->d.C3fix) {
        e = launch_fix_dense(h, X, B, acc, st);
    } else if (e == cudaSuccess && M > 0) {
        const size_t sm = sizeof(uint32_t) * (((size_t)(h->W + 1) * 32 + 1) & ~(size_t)1) +
                          sizeof(long long) * (kFixThreads / 32) * 32;
        if (h->KS == 4)
            energy_fix_kernel<4><<<dim3(tiles, slices), kFixThreads, sm, st>>>(
                X, B, h->N, h->W, h->d.tvars, h->d.tfix, M, per, acc);
        else
            energy_fix_kernel<8><<<dim3(tiles, slices), kFixThreads, sm, st>>>(
                X, B, h->N, h->W, h->d.tvars, h->d.tfix, M, per, acc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        energy_fix_finalize<<<(B + 255) / 256, 256, 0, st>>>(acc, B, h->d.fix_shift, E);
        e = cudaGetLastError();
    }
    cudaFreeAsync(acc, st);
    return e;
}

// The same re-score with caller-owned accumulators: acc must hold B zeroed
// 64-bit words on the device; nothing is allocated here.
cudaError_t launch_energy_fp64_into(const hobo_instance* h, const uint32_t* X, int B, double* E,
                                    unsigned long long* acc, cudaStream_t st)
{
    if (B == 0) return cudaSuccess;
    const int64_t M = h->d.M;
    const int tiles = (B + 31) / 32;
    int slices = (int)std::max<int64_t>(1, std::min<int64_t>((4LL * h->num_sms + tiles - 1) / tiles,
                                                             (M + 4095) / 4096));
    const int64_t per = (M + slices - 1) / std::max(slices, 1);
    cudaError_t e = cudaSuccess;
    if (h->d.C3fix) {
        e = launch_fix_dense(h, X, B, acc, st);
    } else if (M > 0) {
        const size_t sm = sizeof(uint32_t) * (((size_t)(h->W + 1) * 32 + 1) & ~(size_t)1) +
                          sizeof(long long) * (kFixThreads / 32) * 32;
        if (h->KS == 4)
            energy_fix_kernel<4><<<dim3(tiles, slices), kFixThreads, sm, st>>>(
                X, B, h->N, h->W, h->d.tvars, h->d.tfix, M, per, acc);
        else
            energy_fix_kernel<8><<<dim3(tiles, slices), kFixThreads, sm, st>>>(
                X, B, h->N, h->W, h->d.tvars, h->d.tfix, M, per, acc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        energy_fix_finalize<<<(B + 255) / 256, 256, 0, st>>>(acc, B, h->d.fix_shift, E);
        e = cudaGetLastError();
    }
    return e;
}

// ---------------------------------------------------------------------------
// Plain sweep: one thread per state, fields and bits in global memory.
// ---------------------------------------------------------------------------
template <bool DENSE, int KU>
__global__ void sweep_plain_kernel(const SweepDev p)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= p.B) return;
    const int N = p.N, W = p.W, P = p.P;
    float* __restrict__ g = p.g + (int64_t)b * N;
    uint32_t* __restrict__ x = p.X + (int64_t)b * W;
    uint32_t* __restrict__ bx = p.bestX + (int64_t)b * W;
    {
        const int rem = N - 32 * (W - 1);
        if (rem < 32) x[W - 1] &= (1u << rem) - 1u;
    }
    float E = p.E[b], Eb;
    if (p.resume) {
        Eb = p.bestE[b];
    } else {
        Eb = E;
        for (int k = 0; k < W; ++k) bx[k] = x[k];
    }
    long long nacc = 0;
    int64_t nbytes = 0;
    u32x4 r = {0u, 0u, 0u, 0u};
    for (int s = 0; s < p.sweeps; ++s) {
        const float beta = p.beta[s];
        const uint32_t sw = (uint32_t)(p.sweep0 + s);
        for (int i = 0; i < N; ++i) {
            if ((i & 3) == 0)
                r = philox10((uint32_t)(i >> 2), sw, (uint32_t)b, kStreamMetropolis, p.k0, p.k1);
            const uint32_t xi = bit_of(x, i);
            const float gi = g[i];
            const float dE = xi ? -gi : gi;
            if (!metropolis(dE, beta, pick4(r, i & 3))) continue;
            x[i >> 5] ^= 1u << (i & 31);
            E = __fadd_rn(E, dE);
            ++nacc;
            const float delta = xi ? -1.0f : 1.0f;
            if (DENSE) {
                // same sums, in the same order, as the tuned kernel
                const float* slab = p.S3 + (int64_t)i * N * P;
                int pop = 0;
                for (int k = 0; k < W; ++k) pop += __popc(x[k]);
                const bool comp = 2 * pop > N;
                nbytes += (int64_t)(comp ? N - pop : pop) * P * 4 + (comp ? 2 : 1) * (int64_t)P * 4;
                for (int j = 0; j < N; ++j) {
                    float acc = 0.0f;
                    for (int l = 0; l < N; ++l)
                        if (bit_of(x, l) != (comp ? 1u : 0u)) acc = __fadd_rn(acc, slab[(int64_t)l * P + j]);
                    if (comp) acc = __fsub_rn(p.S3col[(int64_t)i * P + j], acc);
                    g[j] = __fadd_rn(g[j], __fmul_rn(delta, __fadd_rn(p.S2[(int64_t)i * P + j], acc)));
                }
            } else {
                // same sums, in the same order, as the tuned kernel
                for (int c = p.cptr[i]; c < p.cptr[i + 1]; ++c) {
                    const int2 hd = p.chdr[c];
                    const int nrec = hd.y & 63;
                    nbytes += 8 + 32 * 4;
                    for (int l = 0; l < nrec; ++l) {
                        const int cnt = p.lcnt[32 * c + l];
                        nbytes += (int64_t)cnt * (4 + 2 * KU);
                        float acc = 0.0f;
                        for (int k = 0; k < cnt; ++k) {
                            const int64_t e = (int64_t)hd.x + 32 * k + l;
                            bool on = true;
                            for (int q = 0; q < KU; ++q) {
                                const int v = p.uconds[e * KU + q];
                                if (v < N && !bit_of(x, v)) on = false;
                            }
                            if (on) acc = __fadd_rn(acc, p.ucoef[e]);
                        }
                        const int j = p.ltgt[32 * c + l];
                        g[j] = __fadd_rn(g[j], __fmul_rn(delta, acc));
                    }
                }
            }
            if (E < Eb) {
                Eb = E;
                for (int k = 0; k < W; ++k) bx[k] = x[k];
            }
        }
    }
    p.E[b] = E;
    p.bestE[b] = Eb;
    if (p.accepts) p.accepts[b] += nacc;
    if (p.coef_bytes) p.coef_bytes[b] += nbytes;
}

SweepDev make_dev(const hobo_instance* h, const SweepArgs& a)
{
    SweepDev p{};
    p.N = h->N; p.W = h->W; p.B = a.B; p.sweeps = a.sweeps; p.sweep0 = a.sweep0;
    p.resume = a.resume; p.P = (h->N + 3) & ~3;
    p.k0 = (uint32_t)a.seed; p.k1 = (uint32_t)(a.seed >> 32);
    p.beta = a.beta; p.X = a.X; p.g = a.g; p.E = a.E; p.bestX = a.bestX; p.bestE = a.bestE;
    p.accepts = a.accepts;
    p.coef_bytes = a.coef_bytes;
    p.write_g = a.write_g ? 1 : 0;
    p.cptr = h->d.cptr; p.chdr = h->d.chdr; p.ltgt = h->d.ltgt; p.lcnt = h->d.lcnt; p.ucoef = h->d.ucoef;
    p.uconds = h->d.uconds; p.S2 = h->d.S2; p.S3 = h->d.S3; p.S3col = h->d.S3col;
    return p;
}

cudaError_t launch_sweep_tuned(const hobo_instance* h, const SweepArgs& a, cudaStream_t st)
{
    if (a.B == 0 || a.sweeps == 0) return cudaSuccess;
    const SweepDev p = make_dev(h, a);
    if (h->dense) return dispatch_tuned<true, 1>(p, st);
    if (h->KU <= 1) return dispatch_tuned<false, 1>(p, st);
    if (h->KU <= 2) return dispatch_tuned<false, 2>(p, st);
    return dispatch_tuned<false, 6>(p, st);
}

cudaError_t launch_sweep_plain(const hobo_instance* h, const SweepArgs& a, cudaStream_t st)
{
    if (a.B == 0 || a.sweeps == 0) return cudaSuccess;
    const SweepDev p = make_dev(h, a);
    const int threads = 128;
    const unsigned grid = (unsigned)((a.B + threads - 1) / threads);
    if (h->dense) sweep_plain_kernel<true, 1><<<grid, threads, 0, st>>>(p);
    else if (h->KU <= 1) sweep_plain_kernel<false, 1><<<grid, threads, 0, st>>>(p);
    else if (h->KU <= 2) sweep_plain_kernel<false, 2><<<grid, threads, 0, st>>>(p);
    else sweep_plain_kernel<false, 6><<<grid, threads, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace hobo
