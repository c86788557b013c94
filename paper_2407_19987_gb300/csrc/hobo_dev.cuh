// Device-side building blocks shared by the library's kernels:
// Philox4x32-10, the fixed-sequence exp2 of the Metropolis test, bit access.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hobo {

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
// ten rounds of two 32x32->64 multiplies whose halves are xored with the
// other counter words and the key; the key is advanced by the Weyl
// constants between rounds.
// ---------------------------------------------------------------------------
struct u32x4 { uint32_t a, b, c, d; };

__device__ __forceinline__ u32x4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

__device__ __forceinline__ uint32_t pick4(const u32x4& r, int k)
{
    return k == 0 ? r.a : (k == 1 ? r.b : (k == 2 ? r.c : r.d));
}

// ---------------------------------------------------------------------------
// exp2 of t <= 0 as a fixed sequence of round-to-nearest float operations
// (no FMA contraction), so that it is reproducible bit for bit by any IEEE
// implementation of the same steps:
//   t < -125 -> 0;  n = floor(t + 1/2);  f = t - n  (|f| <= 1/2)
//   p(f) = sum_{k=0..6} (ln 2)^k / k! * f^k   (Taylor polynomial of 2^f,
//          coefficients rounded to float, Horner order)
//   result = p * 2^n, 2^n assembled in the exponent field (n >= -125 keeps
//   the product normal, so the scaling is exact).
// Relative error against 2^t is below 4e-7 on [-125, 0].  Evaluated without
// branches: arguments below -125 give 0 by a select, so that the 32 lanes
// of a warp never take different paths.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float exp2_fixed(float t)
{
    const bool under = !(t >= -125.0f);
    const float tc = under ? 0.0f : t;
    const float n = floorf(__fadd_rn(tc, 0.5f));
    const float f = __fsub_rn(tc, n);
    float p = __uint_as_float(0x39218489u);                       // (ln2)^6/720
    p = __fadd_rn(__fmul_rn(p, f), __uint_as_float(0x3AAEC3FFu)); // (ln2)^5/120
    p = __fadd_rn(__fmul_rn(p, f), __uint_as_float(0x3C1D955Bu)); // (ln2)^4/24
    p = __fadd_rn(__fmul_rn(p, f), __uint_as_float(0x3D635847u)); // (ln2)^3/6
    p = __fadd_rn(__fmul_rn(p, f), __uint_as_float(0x3E75FDF0u)); // (ln2)^2/2
    p = __fadd_rn(__fmul_rn(p, f), __uint_as_float(0x3F317218u)); // ln2
    p = __fadd_rn(__fmul_rn(p, f), 1.0f);
    const int ni = (int)n;
    const float r = __fmul_rn(p, __uint_as_float((uint32_t)(ni + 127) << 23));
    return under ? 0.0f : r;
}

// Metropolis decision for a float flip delta dE at inverse temperature beta
// with the 32-bit random word w: accept iff dE <= 0 or
// (w >> 8) * 2^-24 < exp2(-(beta*dE) * log2 e).  Evaluated without branches
// (every lane runs the same instructions): for dE <= 0 the argument is
// clamped to 0 (p = 1 > u, the same decision), and no shortcut is taken.
__device__ __forceinline__ bool metropolis(float dE, float beta, uint32_t w)
{
    const float a = __fmul_rn(beta, dE);
    const float t = fminf(-__fmul_rn(a, __uint_as_float(0x3FB8AA3Bu)), 0.0f);   // log2(e)
    const float p = exp2_fixed(t);
    const float u = __fmul_rn((float)(w >> 8), 5.9604644775390625e-8f);  // 2^-24
    return (dE <= 0.0f) | (u < p);
}

// Stream ids of the random counter (fourth counter word).
constexpr uint32_t kStreamMetropolis = 0u;
constexpr uint32_t kStreamInit = 1u;

// Word w of the initial state b: bit i is bit 31 of word (i % 4) of the
// Philox block with counter (i / 4, 0, b, 1); bits >= N are zero.
__device__ __forceinline__ uint32_t init_word(uint32_t b, int w, int N, uint32_t k0, uint32_t k1)
{
    uint32_t word = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const u32x4 r = philox10((uint32_t)(8 * w + q), 0u, b, kStreamInit, k0, k1);
        word |= ((r.a >> 31) << (4 * q)) | ((r.b >> 31) << (4 * q + 1)) |
                ((r.c >> 31) << (4 * q + 2)) | ((r.d >> 31) << (4 * q + 3));
    }
    const int rem = N - 32 * w;
    if (rem < 32) word &= (1u << rem) - 1u;
    return word;
}

__device__ __forceinline__ uint32_t bit_of(const uint32_t* words, int i)
{
    return (words[i >> 5] >> (i & 31)) & 1u;
}

// Status word code a kernel writes when a bounded device-side wait gave up
// (0 = none); hobo_check / hobo_mlp_check report it as HOBO_ERR_TIMEOUT.
constexpr int kDevTimeout = 1;

}  // namespace hobo
