// Result table of a sampling run: the distinct states among the B returned
// states, each with its energy, number of occurrences and first index,
// sorted by energy (the sampler output of Sec. V: states listed by energy
// with occurrence counts), ties by the first index.
//
// Steps, all on the device:
//   1. sort the state indices by (energy, packed words, index): a bitonic
//      network over a power-of-two index array (padding sorts last); one
//      launch per (k, j) stage, the stages with j < 1024 of one k fused in
//      shared memory;
//   2. mark the first index of every run of equal (energy, words): equal
//      states are adjacent, and the run's first entry has the lowest index;
//   3. exclusive scan of the marks (block scan + scan of block sums) gives
//      each run its group number, and the group count K;
//   4. sort the K groups by (energy, first index) with the same network and
//      write the table in that order.
#include <algorithm>
#include <cstring>
#include <string>

#include "hobo_internal.h"

namespace hobo {

struct AggKeys {
    const uint32_t* X;
    const double* E;
    int W;
};

__device__ __forceinline__ uint64_t order_key(double e)
{
    // order-preserving unsigned image of a double (-0 mapped to +0)
    uint64_t u = (uint64_t)__double_as_longlong(e + 0.0);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// a < b for state indices (energy, words, index); -1 is +infinity
__device__ __forceinline__ bool state_less(const AggKeys& k, int a, int b)
{
    if (b < 0) return a >= 0;
    if (a < 0) return false;
    const uint64_t ea = order_key(k.E[a]), eb = order_key(k.E[b]);
    if (ea != eb) return ea < eb;
    const uint32_t* xa = k.X + (int64_t)a * k.W;
    const uint32_t* xb = k.X + (int64_t)b * k.W;
    for (int w = 0; w < k.W; ++w)
        if (xa[w] != xb[w]) return xa[w] < xb[w];
    return a < b;
}

__device__ __forceinline__ bool same_state(const AggKeys& k, int a, int b)
{
    if (order_key(k.E[a]) != order_key(k.E[b])) return false;
    const uint32_t* xa = k.X + (int64_t)a * k.W;
    const uint32_t* xb = k.X + (int64_t)b * k.W;
    for (int w = 0; w < k.W; ++w)
        if (xa[w] != xb[w]) return false;
    return true;
}

// groups: (energy of its representative, first index); -1 is +infinity
struct GroupKeys {
    const double* E;      // input energies
    const int* rep;       // representative (first) index of group g
};

__device__ __forceinline__ bool group_less(const GroupKeys& k, int a, int b)
{
    if (b < 0) return a >= 0;
    if (a < 0) return false;
    const int ra = k.rep[a], rb = k.rep[b];
    const uint64_t ea = order_key(k.E[ra]), eb = order_key(k.E[rb]);
    if (ea != eb) return ea < eb;
    return ra < rb;
}

template <typename Keys, bool (*LESS)(const Keys&, int, int)>
__global__ void bitonic_global_kernel(int* __restrict__ v, int n, int k, int j, Keys keys)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = i ^ j;
    if (p <= i) return;
    const int a = v[i], b = v[p];
    const bool up = (i & k) == 0;
    if (up ? LESS(keys, b, a) : LESS(keys, a, b)) {
        v[i] = b;
        v[p] = a;
    }
}

// all stages j = jmax, jmax/2, ..., 1 of one k inside blocks of 2*jmax
// elements (jmax < 1024: a block of 1024 threads holds 2048 elements)
template <typename Keys, bool (*LESS)(const Keys&, int, int)>
__global__ void bitonic_shared_kernel(int* __restrict__ v, int n, int k, int jmax, Keys keys)
{
    __shared__ int s[2048];
    const int base = blockIdx.x * 2048;
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) s[t] = base + t < n ? v[base + t] : -1;
    __syncthreads();
    for (int j = jmax; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
            const int p = t ^ j;
            if (p > t) {
                const int a = s[t], b = s[p];
                const bool up = ((base + t) & k) == 0;
                if (up ? LESS(keys, b, a) : LESS(keys, a, b)) {
                    s[t] = b;
                    s[p] = a;
                }
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < 2048; t += blockDim.x)
        if (base + t < n) v[base + t] = s[t];
}

template <typename Keys, bool (*LESS)(const Keys&, int, int)>
static cudaError_t bitonic_sort(int* v, int n, const Keys& keys, cudaStream_t st)
{
    // n is a power of two
    for (int k = 2; k <= n; k <<= 1) {
        int j = k >> 1;
        for (; j >= 1024; j >>= 1)
            bitonic_global_kernel<Keys, LESS><<<(n + 255) / 256, 256, 0, st>>>(v, n, k, j, keys);
        if (j > 0) bitonic_shared_kernel<Keys, LESS><<<(n + 2047) / 2048, 1024, 0, st>>>(v, n, k, j, keys);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

__global__ void iota_pad_kernel(int* __restrict__ v, int B, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i < B ? i : -1;
}

__global__ void run_heads_kernel(const int* __restrict__ idx, int B, AggKeys keys, int* __restrict__ head)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < B) head[p] = (p == 0 || !same_state(keys, idx[p], idx[p - 1])) ? 1 : 0;
}

// exclusive scan of 1024-element blocks; block totals to sums
__global__ void scan_blocks_kernel(const int* __restrict__ in, int n, int* __restrict__ out, int* __restrict__ sums)
{
    __shared__ int warp_tot[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int v = i < n ? in[i] : 0;
    int x = v;
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = warp_tot[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, d);
            if (lane >= d) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    const int incl = x + (wid > 0 ? warp_tot[wid - 1] : 0);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == 1023) sums[blockIdx.x] = incl;
}

// exclusive scan of the block sums in place (one block, sequential chunks)
__global__ void scan_sums_kernel(int* __restrict__ sums, int nb)
{
    __shared__ int carry;
    __shared__ int warp_tot[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c0 = 0; c0 < nb; c0 += 1024) {
        const int i = c0 + threadIdx.x;
        const int v = i < nb ? sums[i] : 0;
        int x = v;
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int t = warp_tot[lane];
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, d);
                if (lane >= d) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const int incl = x + (wid > 0 ? warp_tot[wid - 1] : 0);
        const int c = carry;
        if (i < nb) sums[i] = c + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c + incl;
        __syncthreads();
    }
}

// group numbers; per group its start position, representative and the
// group count (last element)
__global__ void group_starts_kernel(const int* __restrict__ head, const int* __restrict__ pre,
                                    const int* __restrict__ sums, const int* __restrict__ idx, int B,
                                    int* __restrict__ start, int* __restrict__ rep, int* __restrict__ K)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= B) return;
    const int g = pre[p] + sums[p >> 10];
    if (head[p]) {
        start[g] = p;
        rep[g] = idx[p];
    }
    if (p == B - 1) *K = g + head[p];
}

__global__ void iota_groups_kernel(int* __restrict__ v, const int* __restrict__ K, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i < *K ? i : -1;
}

__global__ void write_table_kernel(const int* __restrict__ order, const int* __restrict__ K,
                                   const int* __restrict__ start, const int* __restrict__ rep, int B, int W,
                                   const uint32_t* __restrict__ X, const double* __restrict__ E,
                                   uint32_t* __restrict__ U, double* __restrict__ UE, int64_t* __restrict__ count,
                                   int32_t* __restrict__ first)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int Kv = *K;
    if (r >= Kv) return;
    const int g = order[r];
    const int s0 = start[g];
    const int s1 = g + 1 < Kv ? start[g + 1] : B;
    const int b = rep[g];
    for (int w = 0; w < W; ++w) U[(int64_t)r * W + w] = X[(int64_t)b * W + w];
    UE[r] = E[b];
    count[r] = s1 - s0;
    first[r] = b;
}

}  // namespace hobo

using namespace hobo;

extern "C" int hobo_aggregate(int W, const uint32_t* X, const double* E, int B, uint32_t* U, double* UE,
                              int64_t* count, int32_t* first, int32_t* K, void* stream)
{
    if (W < 1 || W > 32) { set_error("W must be 1..32"); return HOBO_ERR_ARG; }
    if (B < 0 || B > (1 << 30)) { set_error("B must be 0..2^30"); return HOBO_ERR_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    if (!K) { set_error("K is NULL"); return HOBO_ERR_ARG; }
    if (B == 0) {
        const cudaError_t e = cudaMemsetAsync(K, 0, sizeof(int32_t), st);
        if (e != cudaSuccess) { set_error(std::string("aggregate: ") + cudaGetErrorString(e)); return HOBO_ERR_CUDA; }
        return HOBO_OK;
    }
    if (!X || !E || !U || !UE || !count || !first) { set_error("NULL argument"); return HOBO_ERR_ARG; }
    int n = 1;
    while (n < B) n <<= 1;
    const int nb = (B + 1023) / 1024;
    int *idx = nullptr, *head = nullptr, *pre = nullptr, *sums = nullptr, *start = nullptr, *rep = nullptr,
        *order = nullptr;
    cudaError_t e = cudaSuccess;
    auto A = [&](int** p, size_t cnt) { if (e == cudaSuccess) e = cudaMallocAsync((void**)p, sizeof(int) * cnt, st); };
    A(&idx, n); A(&head, B); A(&pre, B); A(&sums, nb); A(&start, B); A(&rep, B); A(&order, n);
    AggKeys keys{X, E, W};
    if (e == cudaSuccess) {
        iota_pad_kernel<<<(n + 255) / 256, 256, 0, st>>>(idx, B, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = bitonic_sort<AggKeys, state_less>(idx, n, keys, st);
    if (e == cudaSuccess) {
        run_heads_kernel<<<(B + 255) / 256, 256, 0, st>>>(idx, B, keys, head);
        scan_blocks_kernel<<<nb, 1024, 0, st>>>(head, B, pre, sums);
        scan_sums_kernel<<<1, 1024, 0, st>>>(sums, nb);
        group_starts_kernel<<<(B + 255) / 256, 256, 0, st>>>(head, pre, sums, idx, B, start, rep, K);
        iota_groups_kernel<<<(n + 255) / 256, 256, 0, st>>>(order, K, n);
        e = cudaGetLastError();
    }
    GroupKeys gk{E, rep};
    if (e == cudaSuccess) e = bitonic_sort<GroupKeys, group_less>(order, n, gk, st);
    if (e == cudaSuccess) {
        write_table_kernel<<<(B + 255) / 256, 256, 0, st>>>(order, K, start, rep, B, W, X, E, U, UE, count, first);
        e = cudaGetLastError();
    }
    int* fr[] = {idx, head, pre, sums, start, rep, order};
    for (int* p : fr)
        if (p) cudaFreeAsync(p, st);
    if (e != cudaSuccess) {
        set_error(std::string("aggregate: ") + cudaGetErrorString(e));
        return HOBO_ERR_CUDA;
    }
    set_error("");
    return HOBO_OK;
}
