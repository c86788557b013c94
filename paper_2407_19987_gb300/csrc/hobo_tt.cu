// Tensor-train contraction (Sec. VI): a tensor given by its train of cores
// G_c [r_{c-1}][N][r_c] (r_0 = r_d = 1, Sec. VI's decomposition) is
// contracted with a state x in every slot: E(x) = sum over all index tuples
// of A[i1..id] x_i1 ... x_id = M_1 M_2 ... M_d with M_c = sum_i x_i G_c[:, i, :],
// which costs d * N * r^2 per state instead of N^d.  For binary x and a train
// of a HOBO tensor this is the energy of Sec. II.C.
//
// One warp per state; the row vector v = M_1 ... M_c stays in shared
// memory.  For a core whose slab G_c[:, i, :] has at most 1024 entries the
// warp first forms M_c itself: lane l owns entries l, l+32, ... of the slab
// (stored [i][a][j], contiguous) and adds them over the set bits i in
// ascending order, independent coalesced loads; then v_new[j] = sum_a v[a]
// M_c[a][j] (a ascending).  Larger slabs: lane j accumulates v_new[j] = sum
// over set bits i of sum_a v[a] G_c[a][i][j] directly.  Float32 sums.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "hobo_internal.h"

constexpr int kTtMaxRank = 256;
constexpr int kTtWarps = 4;

struct hobo_tt {
    int order = 0, N = 0, W = 0;
    int ranks[HOBO_MAX_ORDER + 1] = {0};
    int64_t off[HOBO_MAX_ORDER] = {0};
    float* cores = nullptr;   // core c at off[c], stored [N][r_{c-1}][r_c]
};

namespace hobo {

struct TtShape {
    int order, N, W;
    int ranks[HOBO_MAX_ORDER + 1];
    int64_t off[HOBO_MAX_ORDER];
};

__global__ void __launch_bounds__(kTtWarps * 32)
tt_energy_kernel(const uint32_t* __restrict__ X, int B, const float* __restrict__ cores, const TtShape s,
                 float* __restrict__ E)
{
    __shared__ float vbuf[kTtWarps][2][kTtMaxRank];
    __shared__ float mbuf[kTtWarps][1024];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = blockIdx.x * kTtWarps + warp;
    if (b >= B) return;
    float* vin = vbuf[warp][0];
    float* vout = vbuf[warp][1];
    if (lane == 0) vin[0] = 1.0f;
    __syncwarp();
    for (int c = 0; c < s.order; ++c) {
        const int rin = s.ranks[c], rout = s.ranks[c + 1];
        const float* G = cores + s.off[c];
        const int slab = rin * rout;
        if (slab <= 1024) {
            float m[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) m[k] = 0.0f;
            for (int w = 0; w < s.W; ++w) {
                uint32_t bits = __ldg(X + (int64_t)b * s.W + w);
                const int rem = s.N - 32 * w;
                if (rem < 32) bits &= (1u << rem) - 1u;
                while (bits) {
                    const int i = 32 * w + __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const float* Gi = G + (int64_t)i * slab;
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const int e = k * 32 + lane;
                        if (e < slab) m[k] += __ldg(Gi + e);
                    }
                }
            }
            float* M = mbuf[warp];
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int e = k * 32 + lane;
                if (e < slab) M[e] = m[k];
            }
            __syncwarp();
            for (int j = lane; j < rout; j += 32) {
                float t = 0.0f;
                for (int a = 0; a < rin; ++a) t = fmaf(vin[a], M[a * rout + j], t);
                vout[j] = t;
            }
            __syncwarp();
            float* tmp = vin;
            vin = vout;
            vout = tmp;
            continue;
        }
        float acc[kTtMaxRank / 32];
#pragma unroll
        for (int q = 0; q < kTtMaxRank / 32; ++q) acc[q] = 0.0f;
        const int nq = (rout + 31) / 32;
        for (int w = 0; w < s.W; ++w) {
            uint32_t bits = __ldg(X + (int64_t)b * s.W + w);
            const int rem = s.N - 32 * w;
            if (rem < 32) bits &= (1u << rem) - 1u;
            while (bits) {
                const int i = 32 * w + __ffs(bits) - 1;
                bits &= bits - 1u;
                const float* Gi = G + (int64_t)i * rin * rout;
                for (int a = 0; a < rin; ++a) {
                    const float va = vin[a];
                    const float* row = Gi + (int64_t)a * rout;
#pragma unroll
                    for (int q = 0; q < kTtMaxRank / 32; ++q) {
                        const int j = q * 32 + lane;
                        if (q < nq && j < rout) acc[q] = fmaf(va, __ldg(row + j), acc[q]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kTtMaxRank / 32; ++q) {
            const int j = q * 32 + lane;
            if (q < nq && j < rout) vout[j] = acc[q];
        }
        __syncwarp();
        float* t = vin;
        vin = vout;
        vout = t;
    }
    if (lane == 0) E[b] = vin[0];
}

static int tfail(int code, const std::string& msg)
{
    set_error(msg);
    return code;
}

}  // namespace hobo

using namespace hobo;

extern "C" {

static int hobo_tt_create_impl(hobo_tt_h* out, int order, int N, const int* ranks, const float* cores)
{
    if (!out) return tfail(HOBO_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (order < 1 || order > HOBO_MAX_ORDER) return tfail(HOBO_ERR_ORDER, "order must be 1..8");
    if (N < 1 || N > HOBO_MAX_N) return tfail(HOBO_ERR_ARG, "N must be 1..1024");
    if (!ranks || !cores) return tfail(HOBO_ERR_ARG, "NULL ranks or cores");
    if (ranks[0] != 1 || ranks[order] != 1) return tfail(HOBO_ERR_ARG, "ranks[0] and ranks[order] must be 1");
    for (int c = 1; c < order; ++c)
        if (ranks[c] < 1 || ranks[c] > kTtMaxRank) return tfail(HOBO_ERR_ARG, "ranks must be 1..256");
    hobo_tt* t = new (std::nothrow) hobo_tt();
    if (!t) return tfail(HOBO_ERR_OOM, "host allocation");
    t->order = order;
    t->N = N;
    t->W = (N + 31) / 32;
    int64_t total = 0;
    for (int c = 0; c <= order; ++c) t->ranks[c] = ranks[c];
    for (int c = 0; c < order; ++c) {
        t->off[c] = total;
        total += (int64_t)ranks[c] * N * ranks[c + 1];
    }
    // [r_{c-1}][N][r_c] -> [N][r_{c-1}][r_c]
    std::vector<float> dev((size_t)total);
    for (int c = 0; c < order; ++c) {
        const int ri = ranks[c], ro = ranks[c + 1];
        const float* src = cores + t->off[c];
        float* dst = dev.data() + t->off[c];
        for (int a = 0; a < ri; ++a)
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < ro; ++j) {
                    const float v = src[((int64_t)a * N + i) * ro + j];
                    if (!std::isfinite(v)) {
                        delete t;
                        return tfail(HOBO_ERR_ARG, "non-finite core entry");
                    }
                    dst[((int64_t)i * ri + a) * ro + j] = v;
                }
    }
    cudaError_t e = cudaMalloc((void**)&t->cores, sizeof(float) * (size_t)std::max<int64_t>(total, 1));
    if (e == cudaSuccess) e = cudaMemcpy(t->cores, dev.data(), sizeof(float) * (size_t)total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (t->cores) cudaFree(t->cores);
        delete t;
        return tfail(HOBO_ERR_CUDA, std::string("tt create: ") + cudaGetErrorString(e));
    }
    *out = t;
    set_error("");
    return HOBO_OK;
}

int hobo_tt_create(hobo_tt_h* out, int order, int N, const int* ranks, const float* cores)
{
    return hobo::guarded("hobo_tt_create", [&] { return hobo_tt_create_impl(out, order, N, ranks, cores); });
}

void hobo_tt_destroy(hobo_tt_h t)
{
    if (!t) return;
    if (t->cores) cudaFree(t->cores);
    delete t;
}

int hobo_tt_energy(hobo_tt_h t, const uint32_t* X, int B, float* E, void* stream)
{
    if (!t) return tfail(HOBO_ERR_ARG, "NULL train");
    if (B < 0) return tfail(HOBO_ERR_ARG, "negative B");
    if (B == 0) return HOBO_OK;
    if (!X || !E) return tfail(HOBO_ERR_ARG, "NULL X or E");
    TtShape s{};
    s.order = t->order;
    s.N = t->N;
    s.W = t->W;
    for (int c = 0; c <= t->order; ++c) s.ranks[c] = t->ranks[c];
    for (int c = 0; c < t->order; ++c) s.off[c] = t->off[c];
    tt_energy_kernel<<<(unsigned)((B + kTtWarps - 1) / kTtWarps), kTtWarps * 32, 0, (cudaStream_t)stream>>>(
        X, B, t->cores, s, E);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tfail(HOBO_ERR_CUDA, std::string("tt energy: ") + cudaGetErrorString(e));
    return HOBO_OK;
}

}  // extern "C"
