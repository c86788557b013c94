// CUDA-core kernels: random initial states, term-list energy/field
// contraction (float32), float64 re-scoring, and the Metropolis sweeps
// (tuned warp-per-state kernel and the plain thread-per-state kernel).
#include <algorithm>
#include <mutex>
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
                                   uint32_t k0, uint32_t k1, uint32_t state0)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)B * W) return;
    const int b = (int)(tid / W), w = (int)(tid % W);
    X[tid] = init_word(state0 + (uint32_t)b, w, N, k0, k1);
}

cudaError_t launch_init_states(uint32_t* X, int B, int N, int W, uint64_t seed, cudaStream_t st,
                               uint32_t state0)
{
    if (B == 0) return cudaSuccess;
    const int64_t n = (int64_t)B * W;
    const int threads = 256;
    init_states_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
        X, B, N, W, (uint32_t)seed, (uint32_t)(seed >> 32), state0);
    return cudaGetLastError();
}

// ===========================================================================
// Term-list contraction on CUDA cores, in exact fixed point.
//
// Coefficients are the 64-bit integers round(c * 2^S) of the instance's
// monomial and field lists, S chosen so that the sum of all |c| * 2^S stays
// below 2^62: every partial sum is exact, so the result does not depend on
// how the sums are split between threads and blocks, and the float32 (or
// float64) outputs are the sums rounded once.  Integer instances (sum of
// |c| < 2^24) come out exact.
//
// A block holds 32 states, one per lane.  Their bits are transposed into
// column masks in shared memory: bit l of cm[v] is bit v of state b0 + l
// (cm[N] = all ones is the padding sentinel), so the members of a monomial
// are tested for all 32 states with one AND per member.  Blocks with
// blockIdx.y < ES each sum a slice of the monomial list into the energies
// (64-bit atomics into acc); the others take eight variables each (one per
// warp), and warp j sums its field list: g_j = sum of the coefficients of
// the monomials containing j whose other members are all set (Sec. II.C
// energy differentiated in x_j; dE_j = (1 - 2 x_j) g_j).  Lists are read
// 32 records at a time, coalesced, through a per-warp staging buffer.
// ===========================================================================
constexpr int kEfThreads = 256;
constexpr int kEfWarps = kEfThreads / 32;

template <int KV> struct VarRow;
template <> struct VarRow<2> { using T = uint32_t; };
template <> struct VarRow<4> { using T = uint2; };
template <> struct VarRow<8> { using T = uint4; };

template <int KV>
__device__ __forceinline__ int row_var(const typename VarRow<KV>::T& r, int s)
{
    const uint32_t* w = reinterpret_cast<const uint32_t*>(&r);
    return (int)((w[s >> 1] >> ((s & 1) * 16)) & 0xFFFFu);
}

struct EfArgs {
    const uint32_t* X;
    int B, N, W;
    const uint16_t* tvars;
    const long long* tfix;
    int64_t M;
    int64_t per_slice;   // monomials per energy block
    int ES;              // energy blocks per 32 states
    const int64_t* fptr;
    const uint16_t* fvars;
    const long long* ffix;
    int S;               // fixed-point shift
    int flip;            // write dE_j = (1 - 2 x_j) g_j instead of g_j
    float* out_g;        // [B][N] or null
    unsigned long long* acc;   // [B] energy accumulators (zeroed)
};

// Sum of the records rec0..rec1 of a list whose variables are all set, per
// lane (state).  NV variables per record (row width KV), sentinel cm[N].
template <int NV, int KV>
__device__ __forceinline__ long long sum_active(const uint32_t* cm, const uint16_t* __restrict__ vars,
                                                const long long* __restrict__ coef, int64_t rec0,
                                                int64_t rec1, typename VarRow<KV>::T* sv, long long* sc,
                                                int lane)
{
    using Row = typename VarRow<KV>::T;
    const uint32_t lbit = 1u << lane;
    const Row* rows = reinterpret_cast<const Row*>(vars);
    long long s = 0;
    for (int64_t base = rec0; base < rec1; base += 32) {
        const int64_t e = base + lane;
        if (e < rec1) {
            sv[lane] = __ldg(rows + e);
            sc[lane] = __ldg(coef + e);
        }
        __syncwarp();
        const int n = (int)(rec1 - base < 32 ? rec1 - base : 32);
#pragma unroll 4
        for (int q = 0; q < n; ++q) {
            const Row r = sv[q];
            uint32_t m = lbit;
#pragma unroll
            for (int v = 0; v < NV; ++v) m &= cm[row_var<KV>(r, v)];
            if (m) s += sc[q];
        }
        __syncwarp();
    }
    return s;
}

template <int ORDER>
__global__ void __launch_bounds__(kEfThreads)
energy_fields_kernel(const EfArgs a)
{
    constexpr int KF = ORDER - 1;
    constexpr int KV = KF <= 2 ? 2 : (KF <= 4 ? 4 : 8);
    constexpr int KS = ORDER <= 4 ? 4 : 8;
    constexpr int KR = KV > KS ? KV : KS;
    using RowS = typename VarRow<KR>::T;
    __shared__ uint32_t cm[HOBO_MAX_N + 1];
    __shared__ RowS stv[kEfWarps][32];
    __shared__ long long stc[kEfWarps][32];
    __shared__ long long red[kEfWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b0 = blockIdx.x * 32;
    const int nb = min(32, a.B - b0);

    for (int w = warp; w < a.W; w += kEfWarps) {
        const uint32_t word = lane < nb ? a.X[(int64_t)(b0 + lane) * a.W + w] : 0u;
        const int nv = min(32, a.N - 32 * w);
        for (int t = 0; t < nv; ++t) {
            const uint32_t m = __ballot_sync(0xffffffffu, (word >> t) & 1u);
            if (lane == 0) cm[32 * w + t] = m;
        }
    }
    if (threadIdx.x == 0) cm[a.N] = 0xffffffffu;
    __syncthreads();

    if ((int)blockIdx.y < a.ES) {
        const int64_t t0 = (int64_t)blockIdx.y * a.per_slice;
        const int64_t t1 = min(a.M, t0 + a.per_slice);
        const int64_t span = t1 > t0 ? t1 - t0 : 0;
        const int64_t per_warp = ((span + kEfWarps - 1) / kEfWarps + 31) & ~(int64_t)31;
        const int64_t w0 = min(t1, t0 + (int64_t)warp * per_warp);
        const int64_t w1 = min(t1, w0 + per_warp);
        const long long s = sum_active<ORDER, KS>(
            cm, a.tvars, a.tfix, w0, w1, reinterpret_cast<typename VarRow<KS>::T*>(stv[warp]), stc[warp], lane);
        red[warp][lane] = s;
        __syncthreads();
        if (warp == 0 && lane < nb) {
            long long tot = 0;
#pragma unroll
            for (int q = 0; q < kEfWarps; ++q) tot += red[q][lane];
            atomicAdd(a.acc + b0 + lane, (unsigned long long)tot);
        }
        return;
    }
    const int j = ((int)blockIdx.y - a.ES) * kEfWarps + warp;
    if (j >= a.N) return;
    const long long s = sum_active<KF, KV>(cm, a.fvars, a.ffix, a.fptr[j], a.fptr[j + 1],
                                           reinterpret_cast<typename VarRow<KV>::T*>(stv[warp]), stc[warp],
                                           lane);
    if (lane < nb) {
        float g = scalbnf(__ll2float_rn(s), -a.S);
        if (a.flip && ((cm[j] >> lane) & 1u)) g = -g;
        a.out_g[(int64_t)(b0 + lane) * a.N + j] = g;
    }
}

__global__ void energy_fix_finalize_f32(const unsigned long long* __restrict__ acc, int B, int S,
                                        float* __restrict__ E)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) E[b] = scalbnf(__ll2float_rn((long long)acc[b]), -S);
}

// Energies (into zeroed acc) and, with g, fields of B states.
static cudaError_t launch_energy_fields(const hobo_instance* h, const uint32_t* X, int B, float* g, bool flip,
                                        unsigned long long* acc, cudaStream_t st)
{
    if (B == 0) return cudaSuccess;
    const auto& d = h->d;
    const int tiles = (B + 31) / 32;
    const int gslices = g ? (h->N + kEfWarps - 1) / kEfWarps : 0;
    // energy blocks: enough to fill the GPU when there are no field blocks,
    // else about as much work per block as a field block
    int64_t ES;
    if (g) {
        const int64_t per_field_block = std::max<int64_t>(1, d.F * kEfWarps / std::max(h->N, 1));
        ES = (d.M + per_field_block - 1) / per_field_block;
    } else {
        ES = std::min<int64_t>((4LL * h->num_sms + tiles - 1) / tiles, (d.M + 2047) / 2048);
    }
    ES = std::max<int64_t>(1, std::min<int64_t>(ES, 4096));
    EfArgs a;
    a.X = X; a.B = B; a.N = h->N; a.W = h->W;
    a.tvars = d.tvars; a.tfix = d.tfix; a.M = d.M;
    a.per_slice = (d.M + ES - 1) / ES;
    a.ES = (int)ES;
    a.fptr = d.fptr; a.fvars = d.fvars; a.ffix = d.ffix;
    a.S = d.fix_shift; a.flip = flip ? 1 : 0; a.out_g = g; a.acc = acc;
    const dim3 grid(tiles, (unsigned)(ES + gslices));
    switch (h->order) {
        case 1: energy_fields_kernel<1><<<grid, kEfThreads, 0, st>>>(a); break;
        case 2: energy_fields_kernel<2><<<grid, kEfThreads, 0, st>>>(a); break;
        case 3: energy_fields_kernel<3><<<grid, kEfThreads, 0, st>>>(a); break;
        case 4: energy_fields_kernel<4><<<grid, kEfThreads, 0, st>>>(a); break;
        case 5: energy_fields_kernel<5><<<grid, kEfThreads, 0, st>>>(a); break;
        case 6: energy_fields_kernel<6><<<grid, kEfThreads, 0, st>>>(a); break;
        case 7: energy_fields_kernel<7><<<grid, kEfThreads, 0, st>>>(a); break;
        default: energy_fields_kernel<8><<<grid, kEfThreads, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_energy_terms(const hobo_instance* h, const uint32_t* X, int B, float* E,
                                float* g_or_dE, bool flip_out, cudaStream_t st)
{
    if (B == 0) return cudaSuccess;
    unsigned long long* acc = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&acc, sizeof(unsigned long long) * (size_t)B, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (size_t)B, st);
    if (e == cudaSuccess) e = launch_energy_fields(h, X, B, g_or_dE, flip_out, acc, st);
    if (e == cudaSuccess) {
        energy_fix_finalize_f32<<<(B + 255) / 256, 256, 0, st>>>(acc, B, h->d.fix_shift, E);
        e = cudaGetLastError();
    }
    cudaFreeAsync(acc, st);
    return e;
}

// Energies only of a dense instance, exact on the tensor cores (the
// re-score's limb planes, m < j < l), rounded once to float32 like the
// term-list path; cudaErrorNotSupported without those planes.
cudaError_t launch_energy_exact_f32(const hobo_instance* h, const uint32_t* X, int B, float* E, cudaStream_t st)
{
    if (!exact_tc_supported(h)) return cudaErrorNotSupported;
    if (B == 0) return cudaSuccess;
    unsigned long long* acc = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&acc, sizeof(unsigned long long) * (size_t)B, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (size_t)B, st);
    if (e == cudaSuccess) e = launch_energy_exact_tc(h, X, B, acc, st);
    if (e == cudaSuccess) {
        energy_fix_finalize_f32<<<(B + 255) / 256, 256, 0, st>>>(acc, B, h->d.rs_shift, E);
        e = cudaGetLastError();
    }
    cudaFreeAsync(acc, st);
    return e;
}

// ===========================================================================
// float64 re-scoring: the same exact fixed-point energies, rounded once to
// float64 (integer instances exact; otherwise the error is at most
// (number of terms) * 2^-(S+1), below that of a float64 summation).
// ===========================================================================
constexpr int kFixThreads = 256;

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

cudaError_t launch_energy_fp64_into(const hobo_instance* h, const uint32_t* X, int B, double* E,
                                    unsigned long long* acc, cudaStream_t st)
{
    if (B == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    int shift = h->d.fix_shift;
    if (exact_tc_supported(h)) {
        e = launch_energy_exact_tc(h, X, B, acc, st);
        shift = h->d.rs_shift;
    } else if (h->d.C3fix) {
        e = launch_fix_dense(h, X, B, acc, st);
    } else if (h->d.M > 0) {
        e = launch_energy_fields(h, X, B, nullptr, false, acc, st);
    }
    if (e == cudaSuccess) {
        energy_fix_finalize<<<(B + 255) / 256, 256, 0, st>>>(acc, B, shift, E);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_energy_fp64(const hobo_instance* h, const uint32_t* X, int B, double* E,
                               cudaStream_t st)
{
    if (B == 0) return cudaSuccess;
    unsigned long long* acc = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&acc, sizeof(unsigned long long) * (size_t)B, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (size_t)B, st);
    if (e == cudaSuccess) e = launch_energy_fp64_into(h, X, B, E, acc, st);
    cudaFreeAsync(acc, st);
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
                r = philox10((uint32_t)(i >> 2), sw, p.state0 + (uint32_t)b, kStreamMetropolis, p.k0, p.k1);
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
                const float* slab = p.S3 + (int64_t)i * p.NS * P;
                int pop = 0;
                for (int k = 0; k < W; ++k) pop += __popc(x[k]);
                const bool comp = 2 * pop > N;
                // listed bits: set (clear with comp), except i; one row per
                // pair with a listed bit, the pair row when both are
                auto listed = [&](int l) { return l < N && l != i && bit_of(x, l) != (comp ? 1u : 0u); };
                int nrows = 0;
                for (int l = 0; l < N; l += 2) nrows += (listed(l) || listed(l + 1)) ? 1 : 0;
                nbytes += (int64_t)nrows * P * 4 + (comp ? 2 : 1) * (int64_t)P * 4;
                for (int j = 0; j < N; ++j) {
                    float acc = 0.0f;
                    for (int l = 0; l < N; l += 2) {
                        const bool a0 = listed(l), a1 = listed(l + 1);
                        if (a0 && a1) acc = __fadd_rn(acc, slab[(int64_t)(N + l / 2) * P + j]);
                        else if (a0) acc = __fadd_rn(acc, slab[(int64_t)l * P + j]);
                        else if (a1) acc = __fadd_rn(acc, slab[(int64_t)(l + 1) * P + j]);
                    }
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
    p.resume = a.resume; p.P = (h->N + 3) & ~3; p.NS = h->N + (h->N + 1) / 2;
    p.k0 = (uint32_t)a.seed; p.k1 = (uint32_t)(a.seed >> 32);
    p.state0 = a.state0;
    p.beta = a.beta; p.X = a.X; p.g = a.g; p.E = a.E; p.bestX = a.bestX; p.bestE = a.bestE;
    p.accepts = a.accepts;
    p.coef_bytes = a.coef_bytes;
    p.write_g = a.write_g ? 1 : 0;
    p.cptr = h->d.cptr; p.chdr = h->d.chdr; p.ltgt = h->d.ltgt; p.lcnt = h->d.lcnt; p.ucoef = h->d.ucoef;
    p.uconds = h->d.uconds; p.uent = h->d.uent; p.S2 = h->d.S2; p.S3 = h->d.S3; p.S3col = h->d.S3col;
    p.vcache = a.vcache;
    p.vslots = a.vslots;
    return p;
}

// Dense instances run the schedule in two launches: the first twentieth of
// the sweeps (at least kSplitMin, the high-temperature descent where nearly
// every state flips often and the slab reads are L2-bandwidth bound) with
// the plain update, the rest (few flips, often back and forth between a few
// states) with the late-phase sweep: reuse of the last and cached update
// vectors and visits to the bits not frozen only.  The second launch resumes
// from the first one's states, fields and energies in global memory, so the
// result is that of one launch bit for bit.  (Splitting at 1/10 or 1/40 of
// the dense workload's 1000 sweeps measured 1-2 % slower.)
constexpr int kSplitMin = 16;

// Device memory the late-phase vector cache may take in one call.
constexpr size_t kVCacheBytes = 1ull << 30;

// The vector cache comes from a memory pool of the library's own on each
// device that keeps up to kVCacheBytes between calls (the device's default
// pool hands freed memory back at every synchronization, and mapping the
// cache again cost each call a few hundred microseconds).  nullptr when the
// pool cannot be made.  The pool lives as long as the process (a device
// reset would leave its handle stale).
static cudaMemPool_t vcache_pool()
{
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDevices] = {};
    static bool tried[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!tried[dev]) {
        tried[dev] = true;
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
            uint64_t keep = kVCacheBytes;
            (void)cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            pools[dev] = pool;
        }
        (void)cudaGetLastError();
    }
    return pools[dev];
}

cudaError_t launch_sweep_tuned(const hobo_instance* h, const SweepArgs& a, cudaStream_t st)
{
    if (a.B == 0 || a.sweeps == 0) return cudaSuccess;
    const SweepDev p = make_dev(h, a);
    if (h->dense && a.g && a.sweeps > 2 * kSplitMin) {
        const int s1 = std::max(kSplitMin, a.sweeps / 20);
        SweepArgs a1 = a;
        a1.sweeps = s1;
        a1.write_g = true;
        cudaError_t e = dispatch_tuned<true, 1>(make_dev(h, a1), st);
        if (e != cudaSuccess) return e;
        SweepArgs a2 = a;
        a2.beta = a.beta + s1;
        a2.sweeps = a.sweeps - s1;
        a2.sweep0 = a.sweep0 + s1;
        a2.resume = 1;
        // the late launch's vector cache (layouts of up to 8 words); without
        // it the launch computes every vector, with the same results
        // (kVSlots entries per state, fewer when that would pass kVCacheBytes)
        float* vc = nullptr;
        int slots = 0;
        if (h->W <= 8) {
            const size_t entry = sizeof(float) * (size_t)vcache_entry_floats((h->N + 3) & ~3);
            slots = (int)std::min<size_t>(kVSlots, kVCacheBytes / std::max<size_t>(1, entry * (size_t)a.B));
            cudaMemPool_t pool = slots >= 2 ? vcache_pool() : nullptr;
            if (pool && cudaMallocFromPoolAsync((void**)&vc, entry * (size_t)a.B * slots, pool, st) != cudaSuccess) {
                (void)cudaGetLastError();
                vc = nullptr;
            }
            if (slots < 2) vc = nullptr;
        }
        a2.vcache = vc;
        a2.vslots = vc ? slots : 0;
        e = dispatch_tuned_dense_reuse(make_dev(h, a2), st);
        if (vc) {
            const cudaError_t ef = cudaFreeAsync(vc, st);
            if (e == cudaSuccess) e = ef;
        }
        return e;
    }
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
