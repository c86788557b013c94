// Metropolis sweep kernels (included by the sweep translation units).
#pragma once
#include <algorithm>
#include "hobo_internal.h"
#include "hobo_dev.cuh"

namespace hobo {

// ===========================================================================
// Metropolis sweeps.
//
// Both kernels implement the same sequential semantics per state: for each
// sweep s and each bit i = 0..N-1 in order, dE = (1 - 2 x_i) g_i, accept by
// metropolis(dE, beta_s, word(i, s, state)); on accept flip x_i, E += dE,
// and for every monomial containing i and another member j add
// delta * c * (product of the remaining members) to g_j (delta = +1 for a
// 0->1 flip, -1 for 1->0); keep the best state on strict improvement.
// Update sums are formed in the same order in both kernels, so they agree
// bit for bit on every instance, and with the CPU oracle on integer ones.
// ===========================================================================
struct SweepDev {
    int N, W, B, sweeps, sweep0, resume, P;   // P: row pitch of the dense slab
    int NS;              // rows per dense slab: N rows, then ceil(N/2) pair rows
    int write_g;
    uint32_t k0, k1;
    uint32_t state0;     // global index of state 0 (Philox counter offset)
    const float* beta;
    uint32_t* X;
    float* g;
    float* E;
    uint32_t* bestX;
    float* bestE;
    int64_t* accepts;
    int64_t* coef_bytes;
    const int32_t* cptr;
    const int2* chdr;
    const uint16_t* ltgt;
    const uint16_t* lcnt;
    const float* ucoef;
    const uint16_t* uconds;
    const void* uent;    // packed entries (coefficient bits + conditions)
    const float* S2;     // [N][P]
    const float* S3;     // [N][NS][P]: row l < N is S3[i][l], row N + q the sum of rows 2q, 2q + 1
    const float* S3col;  // [N][P] column sums of each slab
    float* vcache;       // late-phase dense sweep: [B][vslots] vector-cache entries, or null
    int vslots;          // entries per state (2..kVSlots) when vcache is set
};

// ---------------------------------------------------------------------------
// Vector cache of the late-phase dense sweep.  The update vector of a flip
// of bit i is a function of i and of the state after the flip (its row list
// and the set/clear choice are), so a state that flips i again from the
// same state gets the same float vector.  Late in a schedule the states
// that still flip mostly cycle through a few states; each keeps its last
// vslots (at most kVSlots) vectors in global memory (entry: a 64-byte header
// -- bit, state words -- and the vector's N floats), found through 32-bit
// tags (a hash of the bit and of the state) held one per lane in registers,
// and verified against the stored header before use; entries are replaced
// first in, first out.
constexpr int kVSlots = 32;

__host__ __device__ constexpr int vcache_entry_floats(int P) { return 16 + P; }

// Hash terms: the state's hash is the xor of vhash_bit(i) over its set bits.
__device__ __forceinline__ uint32_t vhash_bit(int i)
{
    uint32_t v = (uint32_t)i * 0x9E3779B1u + 0x7F4A7C15u;
    v ^= v >> 15;
    v *= 0x2C1B3C6Du;
    v ^= v >> 12;
    v *= 0x297A2D39u;
    return v ^ (v >> 15);
}

__device__ __forceinline__ uint32_t vhash_key(uint32_t h, int i)
{
    uint32_t v = h ^ ((uint32_t)i * 0x85EBCA6Bu + 0xC2B2AE35u);
    v ^= v >> 16;
    v *= 0x7FEB352Du;
    v ^= v >> 15;
    v *= 0x846CA68Bu;
    return v ^ (v >> 16);
}

template <int WMAX>
__device__ __forceinline__ uint32_t sel_word(const uint32_t (&x)[WMAX], int w)
{
    uint32_t r = x[0];
#pragma unroll
    for (int k = 1; k < WMAX; ++k) r = (k == w) ? x[k] : r;
    return r;
}

template <int WMAX>
__device__ __forceinline__ void set_word(uint32_t (&x)[WMAX], int w, uint32_t v)
{
#pragma unroll
    for (int k = 0; k < WMAX; ++k) x[k] = (k == w) ? v : x[k];
}

// ---------------------------------------------------------------------------
// Tuned sweep: one warp per state.  The state's fields live in shared
// memory; its bits are held (identically) in every lane's registers.  Bits
// are visited a word at a time: lane t evaluates the decision for bit
// 32w + t.  Until the first accepted bit f of the word nothing changes, so
// the decisions of bits < f are final; bit f is then applied (fields
// updated by the whole warp) and the word is re-evaluated from f + 1.  This
// is exactly the sequential order of the definition.
// ---------------------------------------------------------------------------
// Warps per CTA of the single-instance sweep.  One-warp CTAs let the block
// scheduler spread the states evenly over the SMs (4096 states are 27 warps
// per SM); measured 17% faster than 8-warp CTAs on the order-4 workload and
// no slower elsewhere.  Asking for 27 resident CTAs per SM (4104 states in
// one wave on 152 SMs) rather than 32 gives a thread 72 registers instead of
// 64, so more of an update's row loads stay in flight (dense workload:
// sweep 18.6 -> 17.9 ms).
constexpr int kTunedWarps = 1;
constexpr int kTunedMinBlocks = 27;

// Dense order<=3 update for a flip of bit i: g_j += delta * (S2[i][j] +
// sum_{l set} S3[i][l][j]).  When more than half of the bits are set the
// slab sum is formed as colsum[i][j] - sum_{l clear} S3[i][l][j] instead, so
// at most N/2 rows are listed; a pair of listed bits (2q, 2q + 1) is read
// as one pre-summed pair row, so about 3/8 N rows are read.  Lanes own 4 consecutive targets in each
// 128-wide chunk (NC chunks); rows are visited in ascending order, 8 at a
// time with their loads in flight together.
// Shared-memory staging of slab rows by cp.async (16 bytes per lane per
// row chunk, each lane later reading back only what it copied itself).
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// STG > 0: each batch reads 8 rows into registers and STG more into the
// warp's staging rows in shared memory (stage, STG x P floats), so that
// 8 + STG rows are in flight per round trip; rows are still added in
// ascending order.
template <int WMAX, int NC, bool CACHE = false, int STG = 0>
__device__ __forceinline__ int64_t dense_update(const SweepDev& p, float* __restrict__ g,
                                                const uint32_t (&x)[WMAX], int i, float delta, int lane,
                                                uint32_t* __restrict__ rows, float* __restrict__ cache = nullptr,
                                                float* __restrict__ stage = nullptr)
{
    const int N = p.N, P = p.P, W = p.W;
    const float* __restrict__ slab = p.S3 + (int64_t)i * p.NS * P;
    int pop = 0;
#pragma unroll
    for (int k = 0; k < WMAX; ++k) pop += __popc(x[k]);
    const bool comp = 2 * pop > N;
    // the listed bits: set bits, or clear bits below N, except bit i (row i
    // is zero); offsets (in floats, within the slab) of the rows to read, one
    // per pair (2q, 2q + 1) with a listed bit, ascending: the pair row where
    // both are listed, else the listed bit's row
    int nrows = 0;
#pragma unroll
    for (int k = 0; k < WMAX; ++k) {
        if (k >= W) break;
        uint32_t u = x[k];
        if (comp) {
            u = ~u;
            const int rem = N - 32 * k;
            if (rem < 32) u &= (1u << rem) - 1u;
        }
        if (k == (i >> 5)) u &= ~(1u << (i & 31));
        const uint32_t any = (u | (u >> 1)) & 0x55555555u;     // at the pair's even bit
        const uint32_t both = u & (u >> 1) & 0x55555555u;
        if ((any >> lane) & 1u) {
            const int l = 32 * k + lane;
            const int row = ((both >> lane) & 1u) ? N + (l >> 1) : (((u >> lane) & 1u) ? l : l + 1);
            rows[nrows + __popc(any & ((1u << lane) - 1u))] = (uint32_t)(row * P);
        }
        nrows += __popc(any);
    }
    __syncwarp();
    const int64_t bytes = (int64_t)nrows * P * 4 + (comp ? 2 : 1) * (int64_t)P * 4;
    // this lane's columns: 4 consecutive targets in each 128-wide chunk
    const float* base[NC];
    bool jv[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        jv[c] = 128 * c + 4 * lane < P;
        base[c] = slab + (jv[c] ? 128 * c + 4 * lane : 0);
    }
    // accumulators as packed float pairs: add.rn.f32x2 rounds each half
    // exactly like a scalar round-to-nearest add
    uint64_t acc[NC][2];
#pragma unroll
    for (int c = 0; c < NC; ++c) { acc[c][0] = 0ull; acc[c][1] = 0ull; }
    int r0 = 0;
    if (STG > 0) {
#pragma unroll 1
        for (; r0 + 8 + STG <= nrows; r0 += 8 + STG) {
#pragma unroll
            for (int t = 0; t < STG; ++t) {
                const uint32_t o = rows[r0 + 8 + t];
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (jv[c]) cp_async16(stage + t * P + 128 * c + 4 * lane, base[c] + o);
            }
            cp_async_commit();
            const uint4 o0 = *reinterpret_cast<const uint4*>(rows + r0);
            const uint4 o1 = *reinterpret_cast<const uint4*>(rows + r0 + 4);
            const uint32_t off[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
            ulonglong2 v[8][NC];
#pragma unroll
            for (int t = 0; t < 8; ++t)
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    v[t][c] = jv[c] ? __ldg(reinterpret_cast<const ulonglong2*>(base[c] + off[t])) : make_ulonglong2(0ull, 0ull);
#pragma unroll
            for (int t = 0; t < 8; ++t)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc[c][0]) : "l"(v[t][c].x));
                    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc[c][1]) : "l"(v[t][c].y));
                }
            cp_async_wait_all();
#pragma unroll
            for (int t = 0; t < STG; ++t)
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const ulonglong2 w = jv[c] ? *reinterpret_cast<const ulonglong2*>(stage + t * P + 128 * c + 4 * lane)
                                               : make_ulonglong2(0ull, 0ull);
                    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc[c][0]) : "l"(w.x));
                    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc[c][1]) : "l"(w.y));
                }
        }
    }
#pragma unroll 1
    for (; r0 + 8 <= nrows; r0 += 8) {
        const uint4 o0 = *reinterpret_cast<const uint4*>(rows + r0);
        const uint4 o1 = *reinterpret_cast<const uint4*>(rows + r0 + 4);
        const uint32_t off[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
        ulonglong2 v[8][NC];
#pragma unroll
        for (int t = 0; t < 8; ++t)
#pragma unroll
            for (int c = 0; c < NC; ++c)
                v[t][c] = jv[c] ? __ldg(reinterpret_cast<const ulonglong2*>(base[c] + off[t])) : make_ulonglong2(0ull, 0ull);
#pragma unroll
        for (int t = 0; t < 8; ++t)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc[c][0]) : "l"(v[t][c].x));
                asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc[c][1]) : "l"(v[t][c].y));
            }
    }
#pragma unroll 1
    for (; r0 < nrows; ++r0) {
        const uint32_t off = rows[r0];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const ulonglong2 v = jv[c] ? __ldg(reinterpret_cast<const ulonglong2*>(base[c] + off)) : make_ulonglong2(0ull, 0ull);
            asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc[c][0]) : "l"(v.x));
            asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc[c][1]) : "l"(v.y));
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int j = 128 * c + 4 * lane;
        if (!jv[c]) continue;
        const float4 s2 = __ldg(reinterpret_cast<const float4*>(p.S2 + (int64_t)i * P + j));
        float4 d = make_float4(__uint_as_float((uint32_t)acc[c][0]), __uint_as_float((uint32_t)(acc[c][0] >> 32)),
                               __uint_as_float((uint32_t)acc[c][1]), __uint_as_float((uint32_t)(acc[c][1] >> 32)));
        if (comp) {
            const float4 cs = __ldg(reinterpret_cast<const float4*>(p.S3col + (int64_t)i * P + j));
            d = make_float4(__fsub_rn(cs.x, d.x), __fsub_rn(cs.y, d.y), __fsub_rn(cs.z, d.z), __fsub_rn(cs.w, d.w));
        }
        const float a4[4] = {d.x, d.y, d.z, d.w};
        const float s4[4] = {s2.x, s2.y, s2.z, s2.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float u = __fadd_rn(s4[q], a4[q]);
            if (j + q < N) g[j + q] = __fadd_rn(g[j + q], __fmul_rn(delta, u));
            if (CACHE && j + q < N) cache[j + q] = u;
        }
    }
    return bytes;
}

// Late-phase reuse of the update vector.  The vector of a flip of bit i,
// u_j = S2[i][j] + (sum over the row list of slab i's rows), does not depend
// on x_i: bit i is never listed, so when the next accepted flip of a state
// is bit i again (no other bit changed in between) and the choice between
// set rows and clear rows is the same, the row list and so the float vector
// are the same, and the state's last vector, kept in shared memory, is
// applied instead of reading the rows again.  With x already flipped:
template <int WMAX>
__device__ __forceinline__ bool dense_comp(const uint32_t (&x)[WMAX], int N)
{
    int pop = 0;
#pragma unroll
    for (int k = 0; k < WMAX; ++k) pop += __popc(x[k]);
    return 2 * pop > N;
}

// Sparse update for a flip of bit i: lanes take the target records of a
// chunk; each sums, in entry order, the coefficients of its entries whose
// conditions are all set.  The entries of a step k of all lanes are adjacent,
// so every load of the chunk is coalesced and independent of the others.
// Entry e of the packed update lists: its coefficient if all its
// conditions' bits are set, else 0.  bb holds the state's bits one per byte
// (bb[N] = 1: the sentinel of unused condition slots), so a condition is
// one shared-memory byte load.
template <int KU>
__device__ __forceinline__ float packed_entry(const SweepDev& p, const uint8_t* __restrict__ bb, int64_t e)
{
    uint32_t pr;
    float cv;
    auto bit = [&](uint32_t v) { return (uint32_t)bb[v]; };
    if (KU <= 2) {
        const uint2 r = __ldg(reinterpret_cast<const uint2*>(p.uent) + e);
        cv = __uint_as_float(r.x);
        pr = bit(r.y & 0xFFFFu);
        if (KU == 2) pr &= bit(r.y >> 16);
    } else {
        const uint4 r = __ldg(reinterpret_cast<const uint4*>(p.uent) + e);
        cv = __uint_as_float(r.x);
        pr = bit(r.y & 0xFFFFu) & bit(r.y >> 16) & bit(r.z & 0xFFFFu) & bit(r.z >> 16) & bit(r.w & 0xFFFFu) &
             bit(r.w >> 16);
    }
    return (pr & 1u) ? cv : 0.0f;
}

template <int KU>
__device__ __forceinline__ int64_t sparse_update(const SweepDev& p, float* __restrict__ g,
                                                 const uint8_t* __restrict__ bb, int i, float delta,
                                                 int lane)
{
    const int c0 = p.cptr[i], c1 = p.cptr[i + 1];
    int64_t entries = 0;
    for (int c = c0; c < c1; ++c) {
        const int2 hd = p.chdr[c];
        const int K = hd.y >> 6, nrec = hd.y & 63;
        const int j = p.ltgt[32 * c + lane];
        const int cnt = p.lcnt[32 * c + lane];
        if (p.coef_bytes) entries += __reduce_add_sync(0xffffffffu, (unsigned)cnt);
        const int64_t e0 = (int64_t)hd.x + lane;
        float acc = 0.0f;
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
            // adding the 0 of an entry whose conditions are not all set
            // changes nothing: acc starts at +0 and is never -0
            if (k < cnt) acc = __fadd_rn(acc, packed_entry<KU>(p, bb, e0 + 32 * k));
        }
        if (lane < nrec) g[j] = __fadd_rn(g[j], __fmul_rn(delta, acc));
    }
    return (int64_t)(c1 - c0) * (8 + 32 * 4) + entries * (4 + 2 * KU);
}


// Lane t's draw for word w of a group of four words whose Philox blocks the
// warp computed together (lane L holds block 8 * (w0 + L / 8) + L % 8): the
// draw of bit i = 32w + t is word (i % 4) of block i / 4, held by lane
// 8 * (w - w0) + t / 4.
__device__ __forceinline__ uint32_t lane_draw(const u32x4& r4, int w, int lane)
{
    const int src = 8 * (w & 3) + (lane >> 2);
    const uint32_t ra = __shfl_sync(0xffffffffu, r4.a, src);
    const uint32_t rb = __shfl_sync(0xffffffffu, r4.b, src);
    const uint32_t rc = __shfl_sync(0xffffffffu, r4.c, src);
    const uint32_t rd = __shfl_sync(0xffffffffu, r4.d, src);
    const int e = lane & 3;
    return e == 0 ? ra : (e == 1 ? rb : (e == 2 ? rc : rd));
}

// True when some draw of a group's blocks is u = 0 (top 24 bits zero);
// warp-uniform.
__device__ __forceinline__ bool group_has_zero_draw(const u32x4& r4)
{
    const bool z = ((r4.a >> 8) == 0u) | ((r4.b >> 8) == 0u) | ((r4.c >> 8) == 0u) | ((r4.d >> 8) == 0u);
    return __any_sync(0xffffffffu, z) != 0;
}

// The Metropolis decision of metropolis() for the active lanes of a warp
// (all 32 lanes call it), evaluating only what some lane needs.  Downhill
// moves (dE <= 0) are accepted without a draw.  For dE > 0 the decision is
// settled without the exp2 in two cases: a word with (w >> 8) = 0 draws
// u = 0, accepted iff p > 0, i.e. iff the exponent t >= -125; and for
// t < -25, p <= 2^0.5 * (1 + 4e-7) * 2^-25 < 2^-24 <= u for every other
// word, a rejection.  So when the group has no zero draw (gz false) and no
// active uphill lane has t >= -25, every decision is known without the
// lanes' draws, and the shuffles that fetch them are skipped; otherwise the
// draws are fetched once per word (rw, have_rw) and the exp2 is evaluated
// when some lane needs it.  Late in a schedule almost every uphill exponent
// is far below -25.  cand: the lane is active and its move is not frozen
// (frozen_uphill).
__device__ __forceinline__ bool metropolis_lazy(float dE, float beta, bool active, bool gz, const u32x4& r4,
                                                int w, int lane, uint32_t& rw, bool& have_rw, bool& cand)
{
    const float a = __fmul_rn(beta, dE);
    const float t = fminf(-__fmul_rn(a, __uint_as_float(0x3FB8AA3Bu)), 0.0f);   // log2(e)
    const bool up = dE > 0.0f;
    cand = active && !(up && t < -125.0f);
    bool need = active && up && !(t < -25.0f);
    bool acc = !up;
    if (gz || __any_sync(0xffffffffu, need)) {
        if (!have_rw) {
            rw = lane_draw(r4, w, lane);
            have_rw = true;
        }
        const bool u0 = (rw >> 8) == 0u;
        acc = !up || (u0 && t >= -125.0f);
        need = need && !u0;
        if (__any_sync(0xffffffffu, need)) {
            const float p = exp2_fixed(t);
            const float u = __fmul_rn((float)(rw >> 8), 5.9604644775390625e-8f);  // 2^-24
            if (need) acc = u < p;
        }
    }
    return active && acc;
}

// An uphill move whose exponent t is below -125: p = 0, rejected whatever
// the draw.  t is non-increasing in beta (both roundings are monotone), so
// with the field unchanged it stays so at any larger beta.
__device__ __forceinline__ bool frozen_uphill(float dE, float beta)
{
    const float a = __fmul_rn(beta, dE);
    const float t = fminf(-__fmul_rn(a, __uint_as_float(0x3FB8AA3Bu)), 0.0f);
    return dE > 0.0f && t < -125.0f;
}

// Shared-memory floats one warp needs for a state of N variables: fields,
// bits and best bits, then the dense update's list of row offsets (read 8 at
// a time); every part a multiple of 16 bytes.
__host__ __device__ constexpr int warp_region_floats(int N, int WMAX)
{
    return 2 * ((N + 3) & ~3) + 4 * (WMAX + 1) + 8;
}

// Longest candidate list the late-phase dense sweep walks instead of
// visiting every bit, in steps of 32 entries.
constexpr int kCandMaxSteps = 3;

// Staging rows of the late-phase dense update (N <= 256: 27 warps of an SM
// then fit in shared memory with them).
__host__ __device__ constexpr int reuse_stage_rows(int WMAX) { return WMAX <= 8 ? 4 : 0; }

// The same plus the last update vector and the staging rows (late-phase
// dense sweep).
__host__ __device__ constexpr int warp_region_floats_reuse(int N, int WMAX)
{
    return warp_region_floats(N, WMAX) + (1 + reuse_stage_rows(WMAX)) * ((N + 3) & ~3);
}

// The whole anneal of state b of the instance described by p, run by one
// warp whose shared-memory region starts at g.
template <int WMAX, bool DENSE, int KU, bool REUSE = false>
__device__ __forceinline__ void anneal_state(const SweepDev& p, int b, float* g, int lane)
{
    const int N = p.N, W = p.W;
    const int NPAD = (N + 3) & ~3;
    uint32_t* bs = reinterpret_cast<uint32_t*>(g + NPAD);   // bits + sentinel (sparse lookups)
    uint32_t* rows = bs + 4 * (WMAX + 1);                   // dense: offsets of the rows to read
    float* ucache = g + warp_region_floats(N, WMAX);        // REUSE: last update vector
    int last_bit = -1;                                      // REUSE: its bit (warp-uniform)
    bool last_comp = false;

    for (int j = lane; j < N; j += 32) g[j] = p.g[(int64_t)b * N + j];
    uint32_t x[WMAX];
    uint32_t* bxs = bs + (WMAX + 1);                    // best bits of this state
#pragma unroll
    for (int k = 0; k < WMAX; ++k) {
        uint32_t v = (k < W) ? p.X[(int64_t)b * W + k] : 0u;
        const int rem = N - 32 * k;
        if (rem <= 0) v = 0u; else if (rem < 32) v &= (1u << rem) - 1u;
        x[k] = v;
    }
    float E = p.E[b], Eb = E;
    for (int k = lane; k < W; k += 32) bxs[k] = p.resume ? p.bestX[(int64_t)b * W + k] : sel_word(x, k);
    if (p.resume) Eb = p.bestE[b];
    const int wsent = N >> 5;
    const uint32_t sent = 1u << (N & 31);
    // sparse: the bits one per byte in the (dense-only) row-list area
    uint8_t* bb = reinterpret_cast<uint8_t*>(rows);
    if (!DENSE) {
        for (int k = lane; k <= W; k += 32) {
            uint32_t v = (k < W) ? sel_word(x, k) : 0u;
            if (k == wsent) v |= sent;
            bs[k] = v;
        }
        for (int v = lane; v <= N; v += 32) bb[v] = v == N ? 1u : (uint8_t)((sel_word(x, v >> 5) >> (v & 31)) & 1u);
    } else {
        // dense: bs holds the words without a sentinel (a word is read from
        // there once per visit instead of selected out of the registers)
        for (int k = lane; k < W; k += 32) bs[k] = sel_word(x, k);
    }
    __syncwarp();

    long long nacc = 0;
    int64_t nbytes = 0;
    float beta_next = p.sweeps > 0 ? __ldg(p.beta) : 0.0f;     // loaded one sweep ahead
    if constexpr (!REUSE) {
    for (int s = 0; s < p.sweeps; ++s) {
        const float beta = beta_next;
        if (s + 1 < p.sweeps) beta_next = __ldg(p.beta + s + 1);
        const uint32_t sw = (uint32_t)(p.sweep0 + s);
        u32x4 r4 = {0u, 0u, 0u, 0u};
        for (int w = 0; w < W; ++w) {
            // the word as it stands (the copy in bs, a sentinel bit masked)
            uint32_t cw = bs[w] & ((!DENSE && w == wsent) ? ~sent : ~0u);
            const int nbits = min(32, N - 32 * w);
            // The draw of bit i = 32w + t is word (i % 4) of the Philox block
            // with counter (i / 4, s, b, 0).  Every fourth word, lane L
            // computes block 8 * (w + L / 8) + L % 8, covering words w..w+3
            // (lane_draw picks a lane's draw out of them).
            if ((w & 3) == 0)
                r4 = philox10((uint32_t)(8 * w + lane), sw, p.state0 + (uint32_t)b, kStreamMetropolis, p.k0, p.k1);
            const uint32_t rw = lane_draw(r4, w, lane);
            int t0 = 0;
            while (true) {
                const int i = 32 * w + lane;
                bool acc = false;
                float dE = 0.0f;
                if (lane >= t0 && lane < nbits) {
                    const float gi = g[i];
                    dE = ((cw >> lane) & 1u) ? -gi : gi;
                    acc = metropolis(dE, beta, rw);
                }
                const uint32_t m = __ballot_sync(0xffffffffu, acc);
                if (m == 0u) break;
                const int f = __ffs(m) - 1;
                const float dEf = __shfl_sync(0xffffffffu, dE, f);
                const float delta = ((cw >> f) & 1u) ? -1.0f : 1.0f;
                cw ^= 1u << f;
                E = __fadd_rn(E, dEf);
                ++nacc;
                set_word(x, w, cw);
                if (DENSE && lane == 0) bs[w] = cw;      // read again after the warp's next __syncwarp
                if (E < Eb) {
                    Eb = E;
                    for (int k = lane; k < W; k += 32) bxs[k] = sel_word(x, k);
                }
                const int fi = 32 * w + f;
                if (DENSE) {
                    nbytes += dense_update<WMAX, (WMAX >= 4 ? WMAX / 4 : 1)>(p, g, x, fi, delta, lane, rows);
                } else {
                    if (lane == 0) {
                        bs[w] = cw | (w == wsent ? sent : 0u);
                        bb[fi] = (uint8_t)((cw >> f) & 1u);
                    }
                    __syncwarp();
                    nbytes += sparse_update<KU>(p, g, bb, fi, delta, lane);
                }
                __syncwarp();
                t0 = f + 1;
                if (t0 >= nbits) break;
            }
        }
    }
    } else {
    // Late-phase sweep (dense: with the vector reuse and cache; sparse: the
    // term-list update).  With the fields fixed, a bit that
    // frozen_uphill finds frozen at some beta is rejected at every larger
    // beta whatever its draw.  The state keeps a candidate list, cl[0, nc):
    // in ascending order, every bit not frozen under the current fields at
    // beta_list.  A sweep at beta >= beta_list with a short list (at most
    // kCandMaxSteps steps of 32) visits only the listed bits: lane k
    // evaluates entry pos + k with its own Philox block, the first accepted
    // entry is applied, the list is rebuilt over all bits from the new
    // fields (cand_rebuild) and the walk goes on after that bit.  Other
    // sweeps visit every bit, word by word, recording the list when nothing
    // flips; when something flipped and the bits scanned after the last flip
    // were mostly frozen, the list is rebuilt at the end.  The decisions are
    // those of visiting every bit.  (rows also holds the update's row list:
    // a rebuild follows every update made while a list is kept.)
    // the list: sixteen-bit bit indices, at the start of the row-list area
    // (dense; rebuilt after every update that overwrites it) or after the
    // state's bytes (sparse)
    uint16_t* const cl = DENSE ? reinterpret_cast<uint16_t*>(rows) : reinterpret_cast<uint16_t*>(bb + ((N + 16) & ~15));
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t st = p.state0 + (uint32_t)b;
    const int ncmax = kCandMaxSteps * 32 < N ? kCandMaxSteps * 32 : N;
    // vector cache: this state's entries, the state's hash (warp-uniform),
    // lane k's tag of entry k, the valid entries and the next entry to fill
    float* const vc = (WMAX <= 8 && p.vcache) ? p.vcache + (size_t)b * p.vslots * vcache_entry_floats(p.P) : nullptr;
    const int vslots = p.vslots;
    uint32_t vh = 0u;
    if (vc) {
        for (int k = 0; k < W; ++k)
            if ((bs[k] >> lane) & 1u) vh ^= vhash_bit(32 * k + lane);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vh ^= __shfl_xor_sync(0xffffffffu, vh, o);
    }
    uint32_t vtag = 0u, vmask = 0u;
    int vfifo = 0;
    int nc = -1;                       // candidates in cl[0, nc); -1: no valid list
    float beta_list = 0.0f;            // the beta the list was made or last pruned at
    // The list for the current fields at beta bt; returns how many entries
    // are <= bit (32 fw + f) (the walk's next position).
    auto cand_rebuild = [&](float bt, int fw, int f) -> int {
        int base = 0, at = 0;
#pragma unroll
        for (int k = 0; k < WMAX; ++k) {
            if (k >= W) break;
            const int nbits = min(32, N - 32 * k);
            const bool active = lane < nbits;
            const float gi = active ? g[32 * k + lane] : 0.0f;
            const float dE = ((bs[k] >> lane) & 1u) ? -gi : gi;
            const bool cand = active && !frozen_uphill(dE, bt);
            const uint32_t m = __ballot_sync(0xffffffffu, cand);
            if (cand) cl[base + __popc(m & lt)] = (uint16_t)(32 * k + lane);
            if (k < fw) at += __popc(m);
            else if (k == fw) at += __popc(m & (f == 31 ? ~0u : ((2u << f) - 1u)));
            base += __popc(m);
        }
        __syncwarp();
        nc = base;
        beta_list = bt;
        return at;
    };
    for (int s = 0; s < p.sweeps; ++s) {
        const float beta = beta_next;
        if (s + 1 < p.sweeps) beta_next = __ldg(p.beta + s + 1);
        const uint32_t sw = (uint32_t)(p.sweep0 + s);
        if (!(beta >= beta_list)) nc = -1;
        const bool cmode = nc >= 0 && nc <= ncmax;     // walk the list this sweep
        int pos = 0, kept = 0;                          // list walk: next entry, entries kept
        int w = 0, t0 = 0;                              // word scan: next bit
        bool flipped = false;
        int ncb = 0, nscan = 0;        // word scan: candidates recorded, bits scanned since the last flip
        int r4g = -1;                  // group whose Philox blocks r4 holds
        u32x4 r4 = {0u, 0u, 0u, 0u};
        bool gz = true;
        int rww = -1;                  // word whose draws rw holds
        uint32_t rw = 0u;
        while (true) {
            int fw, f;                 // the accepted bit (word, bit)
            float dEf;
            if (cmode) {
                if (pos >= nc) break;
                const int k = pos + lane;
                const bool act = k < nc;
                const int c = act ? (int)cl[k] : 0;
                float dE = 0.0f;
                bool acc = false, keep = false;
                if (act) {
                    const float gi = g[c];
                    dE = ((bs[c >> 5] >> (c & 31)) & 1u) ? -gi : gi;
                    const u32x4 r = philox10((uint32_t)(c >> 2), sw, st, kStreamMetropolis, p.k0, p.k1);
                    const int e = c & 3;
                    acc = metropolis(dE, beta, e == 0 ? r.a : (e == 1 ? r.b : (e == 2 ? r.c : r.d)));
                    keep = !frozen_uphill(dE, beta);
                }
                const uint32_t m = __ballot_sync(0xffffffffu, acc);
                if (m == 0u) {
                    // prune: entries now frozen leave the list
                    const uint32_t km = __ballot_sync(0xffffffffu, keep);
                    __syncwarp();
                    if (keep) cl[kept + __popc(km & lt)] = (uint16_t)c;   // at or below its own slot
                    kept += __popc(km);
                    pos += 32;
                    __syncwarp();
                    continue;
                }
                const int l = __ffs(m) - 1;
                const int cf = __shfl_sync(0xffffffffu, c, l);
                dEf = __shfl_sync(0xffffffffu, dE, l);
                fw = cf >> 5;
                f = cf & 31;
            } else {
                if (w >= W) break;
                const uint32_t cw = bs[w] & ((!DENSE && w == wsent) ? ~sent : ~0u);
                const int nbits = min(32, N - 32 * w);
                if ((w >> 2) != r4g) {
                    r4g = w >> 2;
                    r4 = philox10((uint32_t)(32 * r4g + lane), sw, st, kStreamMetropolis, p.k0, p.k1);
                    gz = group_has_zero_draw(r4);
                }
                const bool active = lane >= t0 && lane < nbits;
                float dE = 0.0f;
                if (active) {
                    const float gi = g[32 * w + lane];
                    dE = ((cw >> lane) & 1u) ? -gi : gi;
                }
                bool have_rw = rww == w, cand;
                const bool acc = metropolis_lazy(dE, beta, active, gz, r4, w, lane, rw, have_rw, cand);
                if (have_rw) rww = w;
                const uint32_t m = __ballot_sync(0xffffffffu, acc);
                if (m == 0u) {
                    const uint32_t cm = __ballot_sync(0xffffffffu, cand);
                    if (!flipped && cand) cl[ncb + __popc(cm & lt)] = (uint16_t)(32 * w + lane);
                    ncb += __popc(cm);
                    nscan += nbits - t0;
                    ++w;
                    t0 = 0;
                    continue;
                }
                fw = w;
                f = __ffs(m) - 1;
                dEf = __shfl_sync(0xffffffffu, dE, f);
            }
            // apply the flip of bit 32 fw + f
            const uint32_t cw = (bs[fw] & ((!DENSE && fw == wsent) ? ~sent : ~0u)) ^ (1u << f);
            const float delta = ((cw >> f) & 1u) ? 1.0f : -1.0f;   // +1: the bit went 0 -> 1
            E = __fadd_rn(E, dEf);
            ++nacc;
            set_word(x, fw, cw);
            if (E < Eb) {
                Eb = E;
                for (int k = lane; k < W; k += 32) bxs[k] = sel_word(x, k);
            }
            const int fi = 32 * fw + f;
            __syncwarp();
            if constexpr (!DENSE) {
                if (lane == 0) {
                    bs[fw] = cw | (fw == wsent ? sent : 0u);
                    bb[fi] = (uint8_t)((cw >> f) & 1u);
                }
                __syncwarp();
                nbytes += sparse_update<KU>(p, g, bb, fi, delta, lane);
            } else {
            const bool comp = dense_comp(x, N);
            if (lane == 0) bs[fw] = cw;            // read again after the __syncwarp below
            vh ^= vhash_bit(fi);                   // the hash of the state after the flip
            if (fi == last_bit && comp == last_comp) {
                for (int j = lane; j < N; j += 32) g[j] = __fadd_rn(g[j], __fmul_rn(delta, ucache[j]));
            } else {
                bool hit = false;
                uint32_t kh = 0u;
                if (vc) {
                    kh = vhash_key(vh, fi);
                    const uint32_t m = __ballot_sync(0xffffffffu, lane < vslots && ((vmask >> lane) & 1u) && vtag == kh);
                    if (m) {
                        const float* e = vc + (size_t)(__ffs(m) - 1) * vcache_entry_floats(p.P);
                        const uint32_t* hd = reinterpret_cast<const uint32_t*>(e);
                        // the vector is read together with the header that
                        // verifies it (one round trip), used only if it does
                        float u[WMAX];
#pragma unroll
                        for (int t = 0; t < WMAX; ++t) u[t] = 32 * t + lane < N ? e[16 + 32 * t + lane] : 0.0f;
                        const bool bad = lane <= W && hd[lane] != (lane == 0 ? (uint32_t)fi : sel_word(x, lane - 1));
                        if (__ballot_sync(0xffffffffu, bad) == 0u) {
#pragma unroll
                            for (int t = 0; t < WMAX; ++t) {
                                const int j = 32 * t + lane;
                                if (j < N) {
                                    g[j] = __fadd_rn(g[j], __fmul_rn(delta, u[t]));
                                    ucache[j] = u[t];
                                }
                            }
                            nbytes += (int64_t)(16 + N) * 4;
                            hit = true;
                        }
                    }
                }
                if (!hit) {
                    nbytes += dense_update<WMAX, (WMAX >= 4 ? WMAX / 4 : 1), true, reuse_stage_rows(WMAX)>(
                        p, g, x, fi, delta, lane, rows, ucache, ucache + NPAD);
                    if (vc) {
                        float* e = vc + (size_t)vfifo * vcache_entry_floats(p.P);
                        __syncwarp();                  // ucache: each lane wrote its own columns
                        for (int j = lane; j < N; j += 32) e[16 + j] = ucache[j];
                        if (lane <= W) reinterpret_cast<uint32_t*>(e)[lane] = lane == 0 ? (uint32_t)fi : sel_word(x, lane - 1);
                        if (lane == vfifo) vtag = kh;
                        vmask |= 1u << vfifo;
                        vfifo = vfifo + 1 == vslots ? 0 : vfifo + 1;
                    }
                }
                last_bit = fi;
                last_comp = comp;
            }
            }
            __syncwarp();
            flipped = true;
            if (cmode) {
                pos = cand_rebuild(beta, fw, f);
                kept = pos;
            } else {
                ncb = 0;
                nscan = 0;
                w = fw;
                t0 = f + 1;
                if (t0 >= min(32, N - 32 * w)) {
                    ++w;
                    t0 = 0;
                }
            }
        }
        if (cmode) {
            nc = kept;
            beta_list = beta;
        } else if (!flipped) {
            nc = ncb;
            beta_list = beta;
        } else if (4 * ncb <= nscan + 32) {
            cand_rebuild(beta, -1, 0);
        } else {
            nc = -1;
        }
    }
    }

    for (int k = lane; k < W; k += 32) {
        p.X[(int64_t)b * W + k] = sel_word(x, k);
        p.bestX[(int64_t)b * W + k] = bxs[k];
    }
    if (p.write_g)
        for (int j = lane; j < N; j += 32) p.g[(int64_t)b * N + j] = g[j];
    if (lane == 0) {
        p.E[b] = E;
        p.bestE[b] = Eb;
        if (p.accepts) p.accepts[b] += nacc;
        if (p.coef_bytes) p.coef_bytes[b] += nbytes;
    }
}

template <int WMAX, bool DENSE, int KU, bool REUSE = false>
__global__ void __launch_bounds__(kTunedWarps * 32, kTunedMinBlocks)
sweep_tuned_kernel(const SweepDev p)
{
    extern __shared__ float sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * kTunedWarps + warp;       // state of this warp
    if (b >= p.B) return;                                // warp-uniform; no block barriers below
    const int rf = (REUSE && DENSE) ? warp_region_floats_reuse(p.N, WMAX) : warp_region_floats(p.N, WMAX);
    anneal_state<WMAX, DENSE, KU, REUSE>(p, b, sm + (size_t)warp * rf, lane);
}

// Batched form: a persistent grid whose warps take (instance, state) work
// items from a queue (items sorted by decreasing cost) until it is empty.
// Every item is annealed exactly as the per-instance kernel would (sparse
// items through the late-phase loop, whose candidate lists skip the frozen
// bits: the same decisions; uneven batch 1.67 -> 1.61 s).  The sparse
// update is bound by instruction issue and dependent L2 round trips, so
// sparse groups of up to 256 variables ask for 7 resident 8-warp CTAs per
// SM (40 registers a thread, some spilled; 56 warps): 2.04 s with 6.
template <bool DENSE, int WMAX>
__host__ __device__ constexpr int batch_min_blocks() { return (!DENSE && WMAX <= 8) ? 7 : 1; }

template <int WMAX, bool DENSE, int KU>
__global__ void __launch_bounds__(256, batch_min_blocks<DENSE, WMAX>())
sweep_batch_kernel(const SweepDev* __restrict__ descs, const int2* __restrict__ items, int nitems,
                   int* __restrict__ counter, int region_floats)
{
    extern __shared__ float sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* region = sm + (size_t)warp * region_floats;
    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nitems) break;
        const int2 it = items[item];
        anneal_state<WMAX, DENSE, KU, !DENSE>(descs[it.x], it.y, region, lane);
        __syncwarp();
    }
}

template <int WMAX, bool DENSE, int KU>
inline cudaError_t run_batch(const SweepDev* descs, const int2* items, int nitems, int* counter, int Nmax,
                             int warps, int ctas, cudaStream_t st)
{
    const int rf = warp_region_floats(Nmax, WMAX);
    const size_t sm = sizeof(float) * (size_t)rf * warps;
    auto kern = sweep_batch_kernel<WMAX, DENSE, KU>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<ctas, warps * 32, sm, st>>>(descs, items, nitems, counter, rf);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Learned-proposal sweep.  In a learned sweep each state scores its bits
// with the network's per-sweep score table (a function of the scaled field
// and the bit) at the start of the sweep, then either orders them by
// descending score (ties by index; a bitonic sort of (score, index) keys
// held in registers, 32*WMAX keys per warp) and attempts the first
// ceil(top_frac * N), or attempts the bits whose score is >= threshold in
// index order.  Attempts go 32 at a time with the same Metropolis test and
// random words as the plain sweep; every plain_every-th sweep is a plain
// sweep over all bits in index order (with plain_every <= 1 every sweep is
// plain and the trajectories equal the tuned kernel's).
// Optionally records, for states b < rec_states and sweeps s with
// s % rec_every == 0, the features of every attempted bit at its decision:
// (clamp(beta*g, +-vmax)/8, 2x-1, -ln(beta)/4) and the bit itself.
// ---------------------------------------------------------------------------
struct LearnedDev {
    const float* tables;   // [sweeps][2][G] logits, or null when every sweep is plain
    int G;
    float vmax;
    int plain_every;
    int select;            // 0: descending score, top_frac; 1: score >= threshold
    float top_frac;
    float threshold;
    int rec_every, rec_states;
    float* rec_F;          // [n_rec_sweeps][rec_states][N][3]
    uint8_t* rec_x;        // [n_rec_sweeps][rec_states][N]
};

__host__ __device__ constexpr int learned_region_floats(int N, int WMAX)
{
    return 2 * ((N + 3) & ~3) + 4 * (WMAX + 1) + 8 + ((N + 3) & ~3) + (((N + 3) & ~3) / 2 + 4);
}

// Score of a bit from the sweep's table: linear interpolation over the
// clamped scaled field, row x of the table.
__device__ __forceinline__ float learned_score(const float* tab, const LearnedDev& L, float scale, float bg,
                                               uint32_t xi)
{
    const float v = fminf(fmaxf(bg, -L.vmax), L.vmax);
    const float pos = (v + L.vmax) * scale;
    const int k = min((int)pos, L.G - 2);
    const float fr = pos - (float)k;
    const float* t = tab + xi * L.G;
    return fmaf(fr, t[k + 1] - t[k], t[k]);
}

// Bitonic sort of 32*E keys into descending order; key r of a lane is
// element r*32 + lane.  Strides below 32 exchange between lanes, larger
// ones between registers of a lane.
template <int E>
__device__ __forceinline__ void bitonic_desc(uint64_t (&key)[E], int lane)
{
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int rj = j >> 5;
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    if (r & rj) continue;
                    const int r2 = r | rj;
                    const bool desc = ((r * 32 + lane) & k) == 0;
                    const uint64_t a = key[r], b = key[r2];
                    if ((a < b) == desc) { key[r] = b; key[r2] = a; }
                }
            } else {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const uint64_t o = __shfl_xor_sync(0xffffffffu, key[r], j);
                    const bool desc = ((r * 32 + lane) & k) == 0;
                    const bool lower = (lane & j) == 0;
                    const bool take_max = lower == desc;
                    const uint64_t mx = key[r] > o ? key[r] : o;
                    const uint64_t mn = key[r] > o ? o : key[r];
                    key[r] = take_max ? mx : mn;
                }
            }
        }
    }
}

template <int WMAX, bool DENSE, int KU>
__device__ __forceinline__ void anneal_state_learned(const SweepDev& p, const LearnedDev& L, int b, float* g,
                                                     int lane)
{
    const int N = p.N, W = p.W;
    const int NPAD = (N + 3) & ~3;
    uint32_t* bs = reinterpret_cast<uint32_t*>(g + NPAD);
    uint32_t* bxs = bs + (WMAX + 1);
    uint32_t* rows = bs + 4 * (WMAX + 1);
    float* score = reinterpret_cast<float*>(rows + NPAD + 8);
    uint16_t* order = reinterpret_cast<uint16_t*>(score + NPAD);

    for (int j = lane; j < N; j += 32) g[j] = p.g[(int64_t)b * N + j];
    uint32_t x[WMAX];
#pragma unroll
    for (int k = 0; k < WMAX; ++k) {
        uint32_t v = (k < W) ? p.X[(int64_t)b * W + k] : 0u;
        const int rem = N - 32 * k;
        if (rem <= 0) v = 0u; else if (rem < 32) v &= (1u << rem) - 1u;
        x[k] = v;
    }
    float E = p.E[b], Eb = E;
    for (int k = lane; k < W; k += 32) bxs[k] = p.resume ? p.bestX[(int64_t)b * W + k] : sel_word(x, k);
    if (p.resume) Eb = p.bestE[b];
    const int wsent = N >> 5;
    const uint32_t sent = 1u << (N & 31);
    // sparse: the bits one per byte in the (dense-only) row-list area
    uint8_t* bb = reinterpret_cast<uint8_t*>(rows);
    if (!DENSE) {
        for (int k = lane; k <= W; k += 32) {
            uint32_t v = (k < W) ? sel_word(x, k) : 0u;
            if (k == wsent) v |= sent;
            bs[k] = v;
        }
        for (int v = lane; v <= N; v += 32) bb[v] = v == N ? 1u : (uint8_t)((sel_word(x, v >> 5) >> (v & 31)) & 1u);
    }
    __syncwarp();

    long long nacc = 0;
    int64_t nbytes = 0;
    for (int s = 0; s < p.sweeps; ++s) {
        const float beta = __ldg(p.beta + s);
        const uint32_t sw = (uint32_t)(p.sweep0 + s);
        const bool plain = L.tables == nullptr || L.plain_every <= 1 ||
                           (int)(sw % (uint32_t)L.plain_every) == L.plain_every - 1;
        const bool rec = L.rec_F && b < L.rec_states && (s % L.rec_every) == 0;
        const int64_t rbase = rec ? ((int64_t)(s / L.rec_every) * L.rec_states + b) * N : 0;
        int nvisit = N;
        if (!plain) {
            const float* tab = L.tables + (size_t)s * 2 * L.G;
            const float scale = (float)(L.G - 1) / (2.f * L.vmax);
            if (L.select == 0) {
                // keys: order-preserving bits of the score (+0 for -0), then
                // 0xFFFF - i so that equal scores put the lower index first;
                // padding keys are 0, below every real key
                uint64_t key[WMAX];
#pragma unroll
                for (int r = 0; r < WMAX; ++r) {
                    const int i = r * 32 + lane;
                    key[r] = 0ull;
                    if (i < N) {
                        const float sc = learned_score(tab, L, scale, beta * g[i],
                                                       (sel_word(x, i >> 5) >> (i & 31)) & 1u) + 0.0f;
                        uint32_t u = __float_as_uint(sc);
                        u ^= (u & 0x80000000u) ? 0xFFFFFFFFu : 0x80000000u;
                        key[r] = ((uint64_t)u << 32) | (uint64_t)(0xFFFFu - (uint32_t)i);
                    }
                }
                bitonic_desc<WMAX>(key, lane);
#pragma unroll
                for (int r = 0; r < WMAX; ++r) {
                    const int p = r * 32 + lane;
                    if (p < N) order[p] = (uint16_t)(0xFFFFu - (uint32_t)(key[r] & 0xFFFFu));
                }
                nvisit = max(1, min(N, (int)ceilf(L.top_frac * (float)N)));
            } else {
                int base = 0;
                for (int k0 = 0; k0 < N; k0 += 32) {
                    const int i = k0 + lane;
                    bool take = false;
                    if (i < N)
                        take = learned_score(tab, L, scale, beta * g[i], (sel_word(x, i >> 5) >> (i & 31)) & 1u) >=
                               L.threshold;
                    const uint32_t m = __ballot_sync(0xffffffffu, take);
                    if (take) order[base + __popc(m & ((1u << lane) - 1u))] = (uint16_t)i;
                    base += __popc(m);
                }
                nvisit = base;
            }
            __syncwarp();
        }
        for (int k0 = 0; k0 < nvisit; k0 += 32) {
            const int kk = k0 + lane;
            const bool valid = kk < nvisit;
            const int i = valid ? (plain ? kk : (int)order[kk]) : 0;
            const u32x4 r4 = philox10((uint32_t)(i >> 2), sw, p.state0 + (uint32_t)b, kStreamMetropolis, p.k0, p.k1);
            const uint32_t rw = pick4(r4, i & 3);
            int t0 = 0;
            while (true) {
                bool acc = false;
                float dE = 0.0f, gi = 0.0f;
                uint32_t xi = 0u;
                if (valid && lane >= t0) {
                    gi = g[i];
                    xi = (sel_word(x, i >> 5) >> (i & 31)) & 1u;
                    dE = xi ? -gi : gi;
                    acc = metropolis(dE, beta, rw);
                }
                const uint32_t m = __ballot_sync(0xffffffffu, acc);
                const int f = m ? __ffs(m) - 1 : 32;
                if (rec && valid && lane >= t0 && lane <= f) {
                    const float v = fminf(fmaxf(beta * gi, -L.vmax), L.vmax);
                    L.rec_F[(rbase + i) * 3] = v / 8.f;
                    L.rec_F[(rbase + i) * 3 + 1] = xi ? 1.f : -1.f;
                    L.rec_F[(rbase + i) * 3 + 2] = -logf(fmaxf(beta, 1e-30f)) / 4.f;
                    L.rec_x[rbase + i] = (uint8_t)xi;
                }
                if (m == 0u) break;
                const int fi = __shfl_sync(0xffffffffu, i, f);
                const float dEf = __shfl_sync(0xffffffffu, dE, f);
                const int fw = fi >> 5;
                const uint32_t fm = 1u << (fi & 31);
                const float delta = (sel_word(x, fw) & fm) ? -1.0f : 1.0f;
#pragma unroll
                for (int k = 0; k < WMAX; ++k) x[k] ^= (k == fw) ? fm : 0u;
                E = __fadd_rn(E, dEf);
                ++nacc;
                if (E < Eb) {
                    Eb = E;
                    for (int k = lane; k < W; k += 32) bxs[k] = sel_word(x, k);
                }
                if (DENSE) {
                    nbytes += dense_update<WMAX, (WMAX >= 4 ? WMAX / 4 : 1)>(p, g, x, fi, delta, lane, rows);
                } else {
                    if (lane == 0) {
                        bs[fw] = sel_word(x, fw) | (fw == wsent ? sent : 0u);
                        bb[fi] = (uint8_t)((sel_word(x, fw) >> (fi & 31)) & 1u);
                    }
                    __syncwarp();
                    nbytes += sparse_update<KU>(p, g, bb, fi, delta, lane);
                }
                __syncwarp();
                t0 = f + 1;
                if (t0 >= 32) break;
            }
        }
    }

    for (int k = lane; k < W; k += 32) {
        p.X[(int64_t)b * W + k] = sel_word(x, k);
        p.bestX[(int64_t)b * W + k] = bxs[k];
    }
    if (p.write_g)
        for (int j = lane; j < N; j += 32) p.g[(int64_t)b * N + j] = g[j];
    if (lane == 0) {
        p.E[b] = E;
        p.bestE[b] = Eb;
        if (p.accepts) p.accepts[b] += nacc;
        if (p.coef_bytes) p.coef_bytes[b] += nbytes;
    }
}

// Same launch shape as the tuned sweep: one-warp CTAs, at least 27 resident
// per SM.
template <int WMAX, bool DENSE, int KU>
__global__ void __launch_bounds__(kTunedWarps * 32, kTunedMinBlocks)
sweep_learned_kernel(const SweepDev p, const LearnedDev L)
{
    extern __shared__ float sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * kTunedWarps + warp;
    if (b >= p.B) return;
    anneal_state_learned<WMAX, DENSE, KU>(p, L, b, sm + (size_t)warp * learned_region_floats(p.N, WMAX), lane);
}

template <int WMAX, bool DENSE, int KU>
inline cudaError_t run_learned(const SweepDev& p, const LearnedDev& L, cudaStream_t st)
{
    const size_t sm = sizeof(float) * (size_t)learned_region_floats(p.N, WMAX) * kTunedWarps;
    auto kern = sweep_learned_kernel<WMAX, DENSE, KU>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)((p.B + kTunedWarps - 1) / kTunedWarps), kTunedWarps * 32, sm, st>>>(p, L);
    return cudaGetLastError();
}

template <bool DENSE, int KU>
cudaError_t dispatch_learned(const SweepDev& p, const LearnedDev& L, cudaStream_t st);
template <> cudaError_t dispatch_learned<true, 1>(const SweepDev&, const LearnedDev&, cudaStream_t);
template <> cudaError_t dispatch_learned<false, 1>(const SweepDev&, const LearnedDev&, cudaStream_t);
template <> cudaError_t dispatch_learned<false, 2>(const SweepDev&, const LearnedDev&, cudaStream_t);
template <> cudaError_t dispatch_learned<false, 6>(const SweepDev&, const LearnedDev&, cudaStream_t);

template <int WMAX, bool DENSE, int KU, bool REUSE = false>
inline cudaError_t run_tuned(const SweepDev& p, cudaStream_t st)
{
    const size_t per_warp =
        sizeof(float) * (size_t)((REUSE && DENSE) ? warp_region_floats_reuse(p.N, WMAX) : warp_region_floats(p.N, WMAX));
    const size_t sm = per_warp * kTunedWarps;
    auto kern = sweep_tuned_kernel<WMAX, DENSE, KU, REUSE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;

    const unsigned grid = (unsigned)((p.B + kTunedWarps - 1) / kTunedWarps);
    kern<<<grid, kTunedWarps * 32, sm, st>>>(p);
    return cudaGetLastError();
}


template <bool DENSE, int KU>
cudaError_t dispatch_batch(const SweepDev* descs, const int2* items, int nitems, int* counter, int Nmax,
                           int Wmax, int warps, int ctas, cudaStream_t st);
template <> cudaError_t dispatch_batch<true, 1>(const SweepDev*, const int2*, int, int*, int, int, int, int, cudaStream_t);
template <> cudaError_t dispatch_batch<false, 1>(const SweepDev*, const int2*, int, int*, int, int, int, int, cudaStream_t);
template <> cudaError_t dispatch_batch<false, 2>(const SweepDev*, const int2*, int, int*, int, int, int, int, cudaStream_t);
template <> cudaError_t dispatch_batch<false, 6>(const SweepDev*, const int2*, int, int*, int, int, int, int, cudaStream_t);

template <bool DENSE, int KU>
cudaError_t dispatch_tuned(const SweepDev& p, cudaStream_t st);
// dense slabs, late phase: the tuned sweep with reuse of the last update vector
cudaError_t dispatch_tuned_dense_reuse(const SweepDev& p, cudaStream_t st);
template <> cudaError_t dispatch_tuned<true, 1>(const SweepDev& p, cudaStream_t st);
template <> cudaError_t dispatch_tuned<false, 1>(const SweepDev& p, cudaStream_t st);
template <> cudaError_t dispatch_tuned<false, 2>(const SweepDev& p, cudaStream_t st);
template <> cudaError_t dispatch_tuned<false, 6>(const SweepDev& p, cudaStream_t st);

}  // namespace hobo
