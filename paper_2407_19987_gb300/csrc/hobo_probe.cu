// Measurement and self-check kernels with no counterpart in the paper:
//  - hobo_probe_l2_read: a plain read of a buffer small enough to stay in
//    L2, the denominator of the sweep's L2 roofline (the sweep streams its
//    coefficient slabs out of L2);
//  - hobo_selftest_philox: the library's Philox4x32-10 against the
//    implementation in the CUDA toolkit's cuRAND device header, on the GPU.
#include <curand_philox4x32_x.h>
#include <algorithm>
#include <string>
#include "hobo_internal.h"
#include "hobo_dev.cuh"

namespace hobo {

// Written only when the xor of everything read equals an improbable value,
// so that the loads cannot be optimised away; never read.
static __device__ unsigned int g_probe_sink;

constexpr int kProbeThreads = 256;
constexpr int kProbeUnroll = 8;

// The launch reads the buffer `reps` times as one virtual array of
// n16 * reps 16-byte vectors (virtual index v is vector v mod n16): thread
// tid takes v = tid, tid + T, tid + 2T, ... (T threads), eight loads in
// flight, cached in L2 only.  Consecutive threads read consecutive vectors,
// and since T does not divide n16 in general a CTA reads other lines in
// each pass.  Needs T <= n16 (one wrap-around subtraction per step).
__global__ void __launch_bounds__(kProbeThreads)
l2_read_probe_kernel(const uint4* __restrict__ buf, int64_t n16, int reps)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const int64_t total = n16 * reps;
    uint32_t acc = 0;
    int64_t j = tid;
    for (int64_t v0 = tid; v0 < total; v0 += kProbeUnroll * nthr) {
        uint4 v[kProbeUnroll];
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
            v[u] = v0 + u * nthr < total ? __ldcg(buf + j) : make_uint4(0u, 0u, 0u, 0u);
            j += nthr;
            if (j >= n16) j -= n16;
        }
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    if (acc == 0x9E3779B9u) g_probe_sink = acc;
}

__global__ void philox_selftest_kernel(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                                       int64_t n, uint32_t* __restrict__ ours, uint32_t* __restrict__ ref)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint2 k = make_uint2(key[2 * i], key[2 * i + 1]);
    const u32x4 a = philox10(c.x, c.y, c.z, c.w, k.x, k.y);
    const uint4 b = curand_Philox4x32_10(c, k);
    ours[4 * i] = a.a; ours[4 * i + 1] = a.b; ours[4 * i + 2] = a.c; ours[4 * i + 3] = a.d;
    ref[4 * i] = b.x; ref[4 * i + 1] = b.y; ref[4 * i + 2] = b.z; ref[4 * i + 3] = b.w;
}

}  // namespace hobo

using namespace hobo;

extern "C" int hobo_probe_l2_read(const void* buf, int64_t bytes, int reps, void* stream)
{
    if (!buf || bytes < 16 * kProbeThreads || (bytes & 15) || ((uintptr_t)buf & 15) || reps < 1 || reps > 4096) {
        set_error("hobo_probe_l2_read: need a 16-byte aligned device buffer, bytes a multiple of 16 and at "
                  "least 4096, reps 1..4096");
        return HOBO_ERR_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        const int64_t n16 = bytes / 16;
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(8LL * sms, n16 / kProbeThreads));
        l2_read_probe_kernel<<<(unsigned)blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(
            static_cast<const uint4*>(buf), n16, reps);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error(std::string("hobo_probe_l2_read: ") + cudaGetErrorString(e));
        return HOBO_ERR_CUDA;
    }
    return HOBO_OK;
}

extern "C" int hobo_selftest_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* ours,
                                    uint32_t* ref, void* stream)
{
    if (n < 0 || (n > 0 && (!ctr || !key || !ours || !ref))) {
        set_error("hobo_selftest_philox: bad arguments");
        return HOBO_ERR_ARG;
    }
    if (n == 0) return HOBO_OK;
    philox_selftest_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(ctr, key, n, ours, ref);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("hobo_selftest_philox: ") + cudaGetErrorString(e));
        return HOBO_ERR_CUDA;
    }
    return HOBO_OK;
}
