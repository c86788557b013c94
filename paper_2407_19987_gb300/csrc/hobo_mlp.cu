// Learned flip proposal: a small MLP that scores each bit of a state from
// (scaled local field, bit, temperature), trained on trajectories of the
// plain annealer.  The paper has no counterpart; this is the learned
// proposal of the annealer's tuned form.
//
// Network: 3 -> H -> H -> 1, ReLU hidden layers, logit output, binary
// cross-entropy loss against a 0/1 label.  Parameters are kept as float32
// masters for the optimiser (Adam) and used, in every forward and backward
// pass, rounded to bf16 (the network is a bf16 network; sums are float32).
// Layout of the flat parameter vector (H = hidden width):
//   W1 [H][3] | b1 [H] | W2 [H][H] (row = output unit) | b2 [H] | w3 [H] | b3
// Features of bit i of a state at inverse temperature beta, field g_i:
//   f0 = clamp(beta * g_i, -vmax, vmax) / 8,  f1 = 2 x_i - 1,  f2 = -ln(beta) / 4
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include "hobo_internal.h"
#include "sweep_impl.cuh"

struct hobo_mlp {
    int H = 256;
    int device = 0;
    int64_t nparam = 0;
    float* master = nullptr;   // float32 masters
    float* bf = nullptr;       // bf16-rounded copies (as float), used by the passes
    float* m1 = nullptr;       // Adam first moments
    float* m2 = nullptr;       // Adam second moments
    float* grad = nullptr;     // gradient of the last loss_grad call
    int64_t step = 0;
    // activations of a training pass, grown on demand
    float* act = nullptr;
    int64_t act_rows = 0;
    float* part = nullptr;     // partial sums of the gradient reductions
    size_t part_floats = 0;
    int* status = nullptr;     // device word: a bounded wait of a network kernel gave up
    bool use_tc = false;       // forward passes and score tables on the tensor cores
};

namespace hobo {

struct MlpOff {
    int64_t W1, b1, W2, b2, w3, b3, n;
};

__host__ __device__ inline MlpOff offsets(int H)
{
    MlpOff o;
    o.W1 = 0;
    o.b1 = 3LL * H;
    o.W2 = 4LL * H;
    o.b2 = 4LL * H + (int64_t)H * H;
    o.w3 = 5LL * H + (int64_t)H * H;
    o.b3 = 6LL * H + (int64_t)H * H;
    o.n = o.b3 + 1;
    return o;
}

__global__ void round_bf16_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __bfloat162float(__float2bfloat16_rn(src[i]));
}

// C[M][N] = sum_k A(m,k) B(k,n), float32; A(m,k) = A[m*lda+k] (or A[k*lda+m]
// if ta), B(k,n) = B[k*ldb+n] (or B[n*ldb+k] if tb).  64x64 tiles, 16-deep
// K slices in shared memory, 4x4 outputs per thread, k ascending.  Block z
// sums k in [z * kchunk, (z + 1) * kchunk) into slice z of C (M x ldc apart).
__global__ void __launch_bounds__(256)
sgemm_kernel(const float* __restrict__ A, int lda, bool ta, const float* __restrict__ B, int ldb, bool tb,
             float* __restrict__ C, int ldc, int M, int N, int K, int kchunk)
{
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(K, kb + kchunk);
    C += (int64_t)blockIdx.z * M * ldc;
    float acc[4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += 16) {
        for (int q = threadIdx.x; q < 16 * 64; q += 256) {
            const int kk = q / 64, mm = q % 64;
            const int m = m0 + mm, k = k0 + kk;
            float a = 0.f, bv = 0.f;
            if (m < M && k < ke) a = ta ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
            const int n = n0 + mm;
            if (n < N && k < ke) bv = tb ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n];
            As[kk][mm] = a;
            Bs[kk][mm] = bv;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) C[(int64_t)m * ldc + n] = acc[i][j];
        }
}

static cudaError_t sgemm(const float* A, int lda, bool ta, const float* B, int ldb, bool tb, float* C, int ldc,
                         int M, int N, int K, cudaStream_t st, int splits = 1)
{
    const int kchunk = ((K + splits - 1) / splits + 15) / 16 * 16;
    dim3 grid((N + 63) / 64, (M + 63) / 64, (unsigned)((K + kchunk - 1) / kchunk));
    sgemm_kernel<<<grid, 256, 0, st>>>(A, lda, ta, B, ldb, tb, C, ldc, M, N, K, kchunk);
    return cudaGetLastError();
}

// out[i] = sum over slices z (ascending) of part[z * count + i]
__global__ void sum_slices_kernel(const float* __restrict__ part, int S, int64_t count, float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float s = part[i];
    for (int z = 1; z < S; ++z) s += part[(int64_t)z * count + i];
    out[i] = s;
}

// z1 = W1 f + b1, h1 = relu(z1)
__global__ void layer1_kernel(const float* __restrict__ F, int64_t n, const float* __restrict__ w, int H,
                              float* __restrict__ Z1, float* __restrict__ H1)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * H) return;
    const int64_t r = q / H;
    const int u = (int)(q % H);
    const MlpOff o = offsets(H);
    const float z = fmaf(w[o.W1 + 3 * u + 2], F[r * 3 + 2],
                         fmaf(w[o.W1 + 3 * u + 1], F[r * 3 + 1], fmaf(w[o.W1 + 3 * u], F[r * 3], w[o.b1 + u])));
    Z1[q] = z;
    H1[q] = fmaxf(z, 0.f);
}

// One warp per row: z2 += b2, h2 = relu(z2), logit = w3.h2 + b3; for
// training also dl = (sigmoid(logit) - y) / n, the row loss and
// D2 = dl * w3 * [z2 > 0] (D2 overwrites Z2, H2 is kept).
__global__ void head_kernel(float* __restrict__ Z2, float* __restrict__ H2, int64_t n, const float* __restrict__ w,
                            int H, const float* __restrict__ y, float* __restrict__ logit, float* __restrict__ dl,
                            float* __restrict__ rowloss)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n) return;
    const MlpOff o = offsets(H);
    float s = 0.f;
    for (int v = lane; v < H; v += 32) {
        const float z = Z2[r * H + v] + w[o.b2 + v];
        Z2[r * H + v] = z;
        const float h = fmaxf(z, 0.f);
        if (H2) H2[r * H + v] = h;
        s = fmaf(w[o.w3 + v], h, s);
    }
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    const float out = s + w[o.b3];
    if (lane == 0 && logit) logit[r] = out;
    if (!y) return;
    const float yr = y[r];
    const float sig = 1.f / (1.f + expf(-out));
    const float g = (sig - yr) / (float)n;
    if (lane == 0) {
        dl[r] = g;
        rowloss[r] = (out > 0.f ? out + log1pf(expf(-out)) : log1pf(expf(out))) - yr * out;
    }
    for (int v = lane; v < H; v += 32) Z2[r * H + v] = Z2[r * H + v] > 0.f ? g * w[o.w3 + v] : 0.f;
}

// D1 *= [z1 > 0]
__global__ void relu_mask_kernel(float* __restrict__ D1, const float* __restrict__ Z1, int64_t count)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < count && !(Z1[q] > 0.f)) D1[q] = 0.f;
}

// Column reductions over the rows in two stages (row blocks, then the
// blocks in order): gb1 = sum D1, gW1[u][k] = sum D1[r][u] F[r][k],
// gb2 = sum D2, gw3 = sum dl H2, gb3 = sum dl, loss = sum rowloss / n.
// Stage 1: block (x, z) sums rows [z * rows_per, (z + 1) * rows_per) for
// outputs t = x * 128 + threadIdx.x into part[z][t][0..3]
// (t < H: d, d*F0, d*F1, d*F2; H <= t < 2H: D2, dl*H2; t = 2H: dl, rowloss).
__global__ void reduce_grads_partial_kernel(const float* __restrict__ F, const float* __restrict__ D1,
                                            const float* __restrict__ D2, const float* __restrict__ H2,
                                            const float* __restrict__ dl, const float* __restrict__ rowloss,
                                            int64_t n, int H, int64_t rows_per, float4* __restrict__ part)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > 2 * H) return;
    const int64_t r0 = (int64_t)blockIdx.z * rows_per;
    const int64_t r1 = min(n, r0 + rows_per);
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t < H) {
        for (int64_t r = r0; r < r1; ++r) {
            const float d = D1[r * H + t];
            a.x += d;
            a.y = fmaf(d, F[r * 3], a.y);
            a.z = fmaf(d, F[r * 3 + 1], a.z);
            a.w = fmaf(d, F[r * 3 + 2], a.w);
        }
    } else if (t < 2 * H) {
        const int v = t - H;
        for (int64_t r = r0; r < r1; ++r) {
            a.x += D2[r * H + v];
            a.y = fmaf(dl[r], H2[r * H + v], a.y);
        }
    } else {
        for (int64_t r = r0; r < r1; ++r) {
            a.x += dl[r];
            a.y += rowloss[r];
        }
    }
    part[(int64_t)blockIdx.z * (2 * H + 1) + t] = a;
}

__global__ void reduce_grads_final_kernel(const float4* __restrict__ part, int Z, int64_t n, int H,
                                          float* __restrict__ grad, float* __restrict__ loss)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > 2 * H) return;
    float4 a = part[t];
    for (int z = 1; z < Z; ++z) {
        const float4 b = part[(int64_t)z * (2 * H + 1) + t];
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
    }
    const MlpOff o = offsets(H);
    if (t < H) {
        grad[o.b1 + t] = a.x;
        grad[o.W1 + 3 * t] = a.y;
        grad[o.W1 + 3 * t + 1] = a.z;
        grad[o.W1 + 3 * t + 2] = a.w;
    } else if (t < 2 * H) {
        grad[o.b2 + t - H] = a.x;
        grad[o.w3 + t - H] = a.y;
    } else {
        grad[o.b3] = a.x;
        if (loss) *loss = a.y / (float)n;
    }
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ wbf, float* __restrict__ m1,
                            float* __restrict__ m2, const float* __restrict__ g, int64_t n, float lr, float c1,
                            float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = 0.9f * m1[i] + 0.1f * gi;
    const float b = 0.999f * m2[i] + 0.001f * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float v = w[i] - lr * (a / c1) / (sqrtf(b / c2) + 1e-8f);
    w[i] = v;
    wbf[i] = __bfloat162float(__float2bfloat16_rn(v));
}

static cudaError_t ensure_act(hobo_mlp* m, int64_t n)
{
    if (n <= m->act_rows) return cudaSuccess;
    if (m->act) cudaFree(m->act);
    m->act = nullptr;
    const int64_t rows = std::max<int64_t>(n, 1024);
    // Z1, H1, Z2/D2, H2, D1: 5 x rows x H; dl, logit, rowloss: 3 x rows
    cudaError_t e = cudaMalloc((void**)&m->act, sizeof(float) * (size_t)rows * (5 * (size_t)m->H + 3));
    if (e != cudaSuccess) return e;
    m->act_rows = rows;
    return cudaSuccess;
}

// forward (and, with y, backward) pass with the bf16 weights
static cudaError_t passes(hobo_mlp* m, const float* F, const float* y, int64_t n, float* logit_out,
                          float* loss_out, cudaStream_t st)
{
    const int H = m->H;
    cudaError_t e = ensure_act(m, n);
    if (e != cudaSuccess) return e;
    const int64_t R = m->act_rows;
    float* Z1 = m->act;
    float* H1 = Z1 + R * H;
    float* Z2 = H1 + R * H;
    float* H2 = Z2 + R * H;
    float* D1 = H2 + R * H;
    float* dl = D1 + R * H;
    float* lg = dl + R;
    float* rl = lg + R;
    const MlpOff o = offsets(H);
    const int64_t cnt = n * H;
    layer1_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(F, n, m->bf, H, Z1, H1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Z2 = H1 W2^T
    if ((e = sgemm(H1, H, false, m->bf + o.W2, H, true, Z2, H, (int)n, H, H, st)) != cudaSuccess) return e;
    head_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(Z2, y ? H2 : nullptr, n, m->bf, H, y,
                                                          logit_out ? logit_out : lg, dl, rl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!y) return cudaSuccess;
    float* D2 = Z2;
    // D1 = (D2 W2) masked by z1 > 0
    if ((e = sgemm(D2, H, false, m->bf + o.W2, H, false, D1, H, (int)n, H, H, st)) != cudaSuccess) return e;
    relu_mask_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(D1, Z1, cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // gW2 = D2^T H1, K = n split over up to 32 slices of >= 256 rows, the
    // slices summed in order; the other gradients in row blocks of 256
    const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(32, n / 256));
    const int64_t rows_per = 256;
    const int Z = (int)((n + rows_per - 1) / rows_per);
    const size_t need = std::max((size_t)splits * H * H, (size_t)Z * (2 * H + 1) * 4);
    if (need > m->part_floats) {
        if (m->part) cudaFree(m->part);
        m->part = nullptr;
        m->part_floats = 0;
        if ((e = cudaMalloc((void**)&m->part, sizeof(float) * need)) != cudaSuccess) return e;
        m->part_floats = need;
    }
    if (splits == 1) {
        if ((e = sgemm(D2, H, true, H1, H, false, m->grad + o.W2, H, H, H, (int)n, st)) != cudaSuccess) return e;
    } else {
        if ((e = sgemm(D2, H, true, H1, H, false, m->part, H, H, H, (int)n, st, splits)) != cudaSuccess) return e;
        const int64_t hh = (int64_t)H * H;
        // the kernel may have used fewer slices than asked (16-row chunks)
        const int kchunk = (((int)n + splits - 1) / splits + 15) / 16 * 16;
        const int used = (int)((n + kchunk - 1) / kchunk);
        sum_slices_kernel<<<(unsigned)((hh + 255) / 256), 256, 0, st>>>(m->part, used, hh, m->grad + o.W2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    float4* part4 = reinterpret_cast<float4*>(m->part);
    const unsigned gx = (unsigned)((2 * H + 1 + 127) / 128);
    // (the weight-gradient slices are consumed above before part is reused)
    reduce_grads_partial_kernel<<<dim3(gx, 1, (unsigned)Z), 128, 0, st>>>(F, D1, D2, H2, dl, rl, n, H, rows_per, part4);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    reduce_grads_final_kernel<<<gx, 128, 0, st>>>(part4, Z, n, H, m->grad, loss_out);
    return cudaGetLastError();
}

static uint64_t splitmix(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double normal01(uint64_t& s)
{
    const double u1 = ((splitmix(s) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

static int mfail(int code, const std::string& msg)
{
    set_error(msg);
    return code;
}

}  // namespace hobo

using namespace hobo;

extern "C" {

static int hobo_mlp_create_impl(hobo_mlp_h* out, int hidden, uint64_t seed)
{
    if (!out) return mfail(HOBO_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (hidden < 32 || hidden > 1024 || hidden % 32) return mfail(HOBO_ERR_ARG, "hidden must be a multiple of 32 in 32..1024");
    hobo_mlp* m = new (std::nothrow) hobo_mlp();
    if (!m) return mfail(HOBO_ERR_OOM, "host allocation");
    m->H = hidden;
    m->use_tc = mlp_tc_supported(hidden);
    cudaGetDevice(&m->device);
    const MlpOff o = offsets(hidden);
    m->nparam = o.n;
    std::vector<float> w((size_t)o.n, 0.f);
    uint64_t s = seed;
    for (int64_t i = 0; i < 3LL * hidden; ++i) w[o.W1 + i] = (float)(normal01(s) * std::sqrt(2.0 / 3.0));
    for (int64_t i = 0; i < (int64_t)hidden * hidden; ++i) w[o.W2 + i] = (float)(normal01(s) * std::sqrt(2.0 / hidden));
    for (int64_t i = 0; i < hidden; ++i) w[o.w3 + i] = (float)(normal01(s) * std::sqrt(1.0 / hidden));
    const size_t bytes = sizeof(float) * (size_t)o.n;
    cudaError_t e = cudaMalloc((void**)&m->master, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->bf, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->m1, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->m2, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->grad, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&m->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(m->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(m->master, w.data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m1, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(m->m2, 0, bytes);
    if (e == cudaSuccess) {
        round_bf16_kernel<<<(unsigned)((o.n + 255) / 256), 256>>>(m->master, m->bf, o.n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        hobo_mlp_destroy(m);
        return mfail(HOBO_ERR_CUDA, std::string("mlp create: ") + cudaGetErrorString(e));
    }
    *out = m;
    return HOBO_OK;
}

int hobo_mlp_create(hobo_mlp_h* out, int hidden, uint64_t seed)
{
    return hobo::guarded("hobo_mlp_create", [&] { return hobo_mlp_create_impl(out, hidden, seed); });
}

void hobo_mlp_destroy(hobo_mlp_h m)
{
    if (!m) return;
    void* ptrs[] = {m->master, m->bf, m->m1, m->m2, m->grad, m->act, m->status, m->part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete m;
}

int64_t hobo_mlp_num_params(hobo_mlp_h m) { return m ? m->nparam : -1; }

int hobo_mlp_set_tensor_cores(hobo_mlp_h m, int on)
{
    if (!m) return mfail(HOBO_ERR_ARG, "NULL network");
    if (on && !mlp_tc_supported(m->H))
        return mfail(HOBO_ERR_UNSUPPORTED, "the tensor-core forward pass needs a hidden width of 64..256, a multiple of 64");
    m->use_tc = on != 0;
    return HOBO_OK;
}

int hobo_mlp_check(hobo_mlp_h m, void* stream)
{
    if (!m) return mfail(HOBO_ERR_ARG, "NULL network");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    int v = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&v, m->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return mfail(HOBO_ERR_CUDA, std::string("mlp check: ") + cudaGetErrorString(e));
    if (v != 0) {
        const int zero = 0;
        cudaMemcpy(m->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
        return mfail(HOBO_ERR_TIMEOUT, "a device-side wait of a network kernel gave up");
    }
    return HOBO_OK;
}

int hobo_mlp_get(hobo_mlp_h m, float* host, int rounded)
{
    if (!m || !host) return mfail(HOBO_ERR_ARG, "NULL argument");
    cudaError_t e = cudaMemcpy(host, rounded ? m->bf : m->master, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? HOBO_OK : mfail(HOBO_ERR_CUDA, "mlp get");
}

int hobo_mlp_set(hobo_mlp_h m, const float* host)
{
    if (!m || !host) return mfail(HOBO_ERR_ARG, "NULL argument");
    for (int64_t i = 0; i < m->nparam; ++i)
        if (!std::isfinite(host[i])) return mfail(HOBO_ERR_ARG, "non-finite weight");
    cudaError_t e = cudaMemcpy(m->master, host, sizeof(float) * m->nparam, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        round_bf16_kernel<<<(unsigned)((m->nparam + 255) / 256), 256>>>(m->master, m->bf, m->nparam);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    m->step = 0;
    if (e == cudaSuccess) e = cudaMemset(m->m1, 0, sizeof(float) * m->nparam);
    if (e == cudaSuccess) e = cudaMemset(m->m2, 0, sizeof(float) * m->nparam);
    return e == cudaSuccess ? HOBO_OK : mfail(HOBO_ERR_CUDA, "mlp set");
}

int hobo_mlp_forward(hobo_mlp_h m, const float* F, int64_t n, float* logit, void* stream)
{
    if (!m || n < 0 || (n > 0 && (!F || !logit))) return mfail(HOBO_ERR_ARG, "bad mlp forward arguments");
    if (n == 0) return HOBO_OK;
    cudaError_t e = m->use_tc ? launch_mlp_forward_tc(m->bf, m->H, n, F, nullptr, 0, 0.f, logit, m->status,
                                                      (cudaStream_t)stream)
                              : passes(m, F, nullptr, n, logit, nullptr, (cudaStream_t)stream);
    return e == cudaSuccess ? HOBO_OK : mfail(HOBO_ERR_CUDA, std::string("mlp forward: ") + cudaGetErrorString(e));
}

int hobo_mlp_loss_grad(hobo_mlp_h m, const float* F, const float* y, int64_t n, float* grad, float* loss, void* stream)
{
    if (!m || n <= 0 || !F || !y) return mfail(HOBO_ERR_ARG, "bad mlp loss_grad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = passes(m, F, y, n, nullptr, loss, st);
    if (e == cudaSuccess && grad)
        e = cudaMemcpyAsync(grad, m->grad, sizeof(float) * m->nparam, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? HOBO_OK : mfail(HOBO_ERR_CUDA, std::string("mlp loss_grad: ") + cudaGetErrorString(e));
}

int hobo_mlp_train_step(hobo_mlp_h m, const float* F, const float* y, int64_t n, float lr, float* loss, void* stream)
{
    if (!m || n <= 0 || !F || !y || !(lr > 0.f)) return mfail(HOBO_ERR_ARG, "bad mlp train_step arguments");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = passes(m, F, y, n, nullptr, loss, st);
    if (e == cudaSuccess) {
        m->step += 1;
        const float c1 = 1.f - std::pow(0.9f, (float)m->step);
        const float c2 = 1.f - std::pow(0.999f, (float)m->step);
        adam_kernel<<<(unsigned)((m->nparam + 255) / 256), 256, 0, st>>>(m->master, m->bf, m->m1, m->m2, m->grad,
                                                                         m->nparam, lr, c1, c2);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HOBO_OK : mfail(HOBO_ERR_CUDA, std::string("mlp train_step: ") + cudaGetErrorString(e));
}

// Checkpoint: a one-line JSON header, then the bf16 weights (little-endian
// uint16, flat layout above).
static int hobo_mlp_save_impl(hobo_mlp_h m, const char* path)
{
    if (!m || !path) return mfail(HOBO_ERR_ARG, "NULL argument");
    std::vector<float> w((size_t)m->nparam);
    if (cudaMemcpy(w.data(), m->master, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost) != cudaSuccess)
        return mfail(HOBO_ERR_CUDA, "mlp save");
    FILE* f = std::fopen(path, "wb");
    if (!f) return mfail(HOBO_ERR_ARG, std::string("cannot open ") + path);
    std::fprintf(f, "{\"format\": \"hobo-mlp-bf16\", \"hidden\": %d, \"params\": %lld, \"inputs\": 3}\n", m->H,
                 (long long)m->nparam);
    std::vector<uint16_t> b((size_t)m->nparam);
    for (int64_t i = 0; i < m->nparam; ++i) {
        __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
        std::memcpy(&b[i], &h, 2);
    }
    const size_t wr = std::fwrite(b.data(), 2, b.size(), f);
    std::fclose(f);
    return wr == b.size() ? HOBO_OK : mfail(HOBO_ERR_ARG, "short write");
}

int hobo_mlp_save(hobo_mlp_h m, const char* path)
{
    return hobo::guarded("hobo_mlp_save", [&] { return hobo_mlp_save_impl(m, path); });
}

static int hobo_mlp_load_impl(hobo_mlp_h* out, const char* path)
{
    if (!out || !path) return mfail(HOBO_ERR_ARG, "NULL argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return mfail(HOBO_ERR_ARG, std::string("cannot open ") + path);
    char line[512] = {0};
    if (!std::fgets(line, sizeof(line), f)) { std::fclose(f); return mfail(HOBO_ERR_ARG, "empty file"); }
    int H = 0;
    long long np = 0;
    const char* ph = std::strstr(line, "\"hidden\":");
    const char* pp = std::strstr(line, "\"params\":");
    if (!std::strstr(line, "hobo-mlp-bf16") || !ph || !pp || std::sscanf(ph + 9, "%d", &H) != 1 ||
        std::sscanf(pp + 9, "%lld", &np) != 1) {
        std::fclose(f);
        return mfail(HOBO_ERR_ARG, "not a hobo-mlp-bf16 file");
    }
    hobo_mlp_h m = nullptr;
    int rc = hobo_mlp_create(&m, H, 0);
    if (rc) { std::fclose(f); return rc; }
    if (np != m->nparam) { std::fclose(f); hobo_mlp_destroy(m); return mfail(HOBO_ERR_ARG, "parameter count mismatch"); }
    std::vector<uint16_t> b((size_t)np);
    const size_t rd = std::fread(b.data(), 2, b.size(), f);
    std::fclose(f);
    if (rd != b.size()) { hobo_mlp_destroy(m); return mfail(HOBO_ERR_ARG, "truncated file"); }
    std::vector<float> w((size_t)np);
    for (int64_t i = 0; i < np; ++i) {
        const uint32_t u = (uint32_t)b[i] << 16;
        std::memcpy(&w[i], &u, 4);
    }
    rc = hobo_mlp_set(m, w.data());
    if (rc) { hobo_mlp_destroy(m); return rc; }
    *out = m;
    return HOBO_OK;
}

int hobo_mlp_load(hobo_mlp_h* out, const char* path)
{
    return hobo::guarded("hobo_mlp_load", [&] { return hobo_mlp_load_impl(out, path); });
}

}  // extern "C"

namespace hobo {

// Score tables of the learned sweep: for sweep s, table[s][x][k] = logit of
// the features (v_k, 2x-1, -ln(beta_s)/4), v_k = -vmax + 2 vmax k/(G-1), the
// scaled field in units of 1/8 after clamping.  Filled by one forward pass.
__global__ void table_features_kernel(const float* __restrict__ beta, int S, int G, float vmax, float* __restrict__ F)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)S * 2 * G) return;
    const int s = (int)(q / (2 * G));
    const int x = (int)((q / G) % 2);
    const int k = (int)(q % G);
    const float v = -vmax + 2.f * vmax * (float)k / (float)(G - 1);
    F[q * 3] = v / 8.f;
    F[q * 3 + 1] = x ? 1.f : -1.f;
    F[q * 3 + 2] = -logf(fmaxf(beta[s], 1e-30f)) / 4.f;
}

cudaError_t mlp_tables(hobo_mlp* m, const float* beta, int S, int G, float vmax, float* tables, float* scratchF,
                       int* status, cudaStream_t st)
{
    const int64_t rows = (int64_t)S * 2 * G;
    if (m->use_tc) return launch_mlp_forward_tc(m->bf, m->H, rows, nullptr, beta, G, vmax, tables, status, st);
    table_features_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(beta, S, G, vmax, scratchF);
    cudaError_t e = cudaGetLastError();
    // forward passes over slices of rows bound the activation memory
    const int64_t chunk = 65536;
    for (int64_t r0 = 0; r0 < rows && e == cudaSuccess; r0 += chunk)
        e = passes(m, scratchF + r0 * 3, nullptr, std::min(chunk, rows - r0), tables + r0, nullptr, st);
    return e;
}

// label of a recorded attempt: 1 if the bit then differs from the state's
// final best state, 0 if it equals it; -1 for a bit that was not attempted
// in that sweep (rec_x still holds the 0xFF fill)
__global__ void record_labels_kernel(const uint8_t* __restrict__ rec_x, const uint32_t* __restrict__ bestX,
                                     int64_t nrec, int rec_states, int N, int W, float* __restrict__ rec_y)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nrec) return;
    const int i = (int)(q % N);
    const int b = (int)((q / N) % rec_states);
    const uint32_t best = (bestX[(int64_t)b * W + (i >> 5)] >> (i & 31)) & 1u;
    const uint8_t xr = rec_x[q];
    rec_y[q] = xr == 0xFF ? -1.f : ((xr != best) ? 1.f : 0.f);
}

SweepDev make_dev(const hobo_instance* h, const SweepArgs& a);

}  // namespace hobo

extern "C" int hobo_anneal_learned(hobo_h h, hobo_mlp_h m, uint64_t seed, int B, const float* beta, int sweeps,
                                   uint32_t* bestX, double* bestE, const hobo_learned_opts* opts, void* stream)
{
    using namespace hobo;
    if (!h) return mfail(HOBO_ERR_ARG, "NULL instance");
    if (B < 0 || sweeps < 0) return mfail(HOBO_ERR_ARG, "negative B or sweeps");
    if (B == 0) return HOBO_OK;
    if (!bestX || !bestE || (sweeps > 0 && !beta)) return mfail(HOBO_ERR_ARG, "NULL bestX/bestE/beta");
    if (h->W > 8) return mfail(HOBO_ERR_UNSUPPORTED, "the learned sweep supports N <= 256");
    for (int s = 0; s < sweeps; ++s)
        if (!(beta[s] >= 0.0f) || !std::isfinite(beta[s])) return mfail(HOBO_ERR_ARG, "beta must be finite and >= 0");
    hobo_learned_opts o{};
    if (opts) o = *opts;
    if (o.plain_every == 0) o.plain_every = 4;
    if (o.select != HOBO_SELECT_ORDER && o.select != HOBO_SELECT_THRESHOLD)
        return mfail(HOBO_ERR_ARG, "select must be HOBO_SELECT_ORDER or HOBO_SELECT_THRESHOLD");
    if (!std::isfinite(o.threshold)) return mfail(HOBO_ERR_ARG, "threshold must be finite");
    if (!(o.top_frac > 0.f)) o.top_frac = 1.f;
    if (o.top_frac > 1.f) o.top_frac = 1.f;
    if (o.table_size == 0) o.table_size = 256;
    if (!(o.vmax > 0.f)) o.vmax = 32.f;
    if (o.table_size < 2 || o.table_size > (1 << 16)) return mfail(HOBO_ERR_ARG, "table_size must be 2..65536");
    const bool record = o.rec_every > 0 && o.rec_states > 0;
    if (record && (!o.rec_F || !o.rec_y)) return mfail(HOBO_ERR_ARG, "recording needs rec_F and rec_y");
    const bool learned = m && o.plain_every > 1;
    cudaStream_t st = (cudaStream_t)stream;
    const int N = h->N, W = h->W, G = o.table_size;
    const int rec_states = std::min(o.rec_states, B);
    const int64_t nrec_sweeps = record ? (sweeps + o.rec_every - 1) / o.rec_every : 0;
    const int64_t nrec = nrec_sweeps * rec_states * N;

    float *d_beta = nullptr, *d_g = nullptr, *d_E = o.E_out, *d_bE = nullptr, *tables = nullptr, *tf = nullptr;
    uint32_t* d_X = o.X_out;
    uint8_t* rx = nullptr;
    bool ownX = false, ownE = false;
    int rc = HOBO_OK;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMallocAsync(p, std::max<size_t>(bytes, 4), st); };
    A((void**)&d_beta, sizeof(float) * std::max(sweeps, 1));
    if (!d_X) { A((void**)&d_X, sizeof(uint32_t) * (size_t)B * W); ownX = true; }
    if (!d_E) { A((void**)&d_E, sizeof(float) * (size_t)B); ownE = true; }
    A((void**)&d_g, sizeof(float) * (size_t)B * N);
    A((void**)&d_bE, sizeof(float) * (size_t)B);
    if (learned) {
        A((void**)&tables, sizeof(float) * (size_t)std::max(sweeps, 1) * 2 * G);
        if (!m->use_tc) A((void**)&tf, sizeof(float) * (size_t)std::max(sweeps, 1) * 2 * G * 3);
    }
    if (record) A((void**)&rx, (size_t)std::max<int64_t>(nrec, 1));
    if (e == cudaSuccess && record) e = cudaMemsetAsync(rx, 0xFF, (size_t)std::max<int64_t>(nrec, 1), st);
    if (e == cudaSuccess && sweeps > 0)
        e = cudaMemcpyAsync(d_beta, beta, sizeof(float) * sweeps, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_init_states(d_X, B, N, W, seed, st);
    if (e == cudaSuccess) rc = energy_dispatch(h, d_X, B, d_E, d_g, false, 0, st);
    if (e == cudaSuccess && rc == HOBO_OK && o.ev_begin) e = cudaEventRecord((cudaEvent_t)o.ev_begin, st);
    if (e == cudaSuccess && rc == HOBO_OK && learned && sweeps > 0)
        e = mlp_tables(m, d_beta, sweeps, G, o.vmax, tables, tf, h->status, st);
    if (e == cudaSuccess && rc == HOBO_OK && sweeps > 0) {
        SweepArgs a;
        a.B = B; a.sweeps = sweeps; a.seed = seed; a.beta = d_beta;
        a.X = d_X; a.g = d_g; a.E = d_E; a.bestX = bestX; a.bestE = d_bE; a.accepts = o.accepts;
        const SweepDev p = make_dev(h, a);
        LearnedDev L{};
        L.tables = learned ? tables : nullptr;
        L.G = G;
        L.vmax = o.vmax;
        L.plain_every = learned ? o.plain_every : 1;
        L.top_frac = o.top_frac;
        L.select = o.select;
        L.threshold = o.threshold;
        L.rec_every = record ? o.rec_every : 1;
        L.rec_states = record ? rec_states : 0;
        L.rec_F = record ? o.rec_F : nullptr;
        L.rec_x = rx;
        if (h->dense) e = dispatch_learned<true, 1>(p, L, st);
        else if (h->KU <= 1) e = dispatch_learned<false, 1>(p, L, st);
        else if (h->KU <= 2) e = dispatch_learned<false, 2>(p, L, st);
        else e = dispatch_learned<false, 6>(p, L, st);
    } else if (e == cudaSuccess && rc == HOBO_OK) {
        e = cudaMemcpyAsync(bestX, d_X, sizeof(uint32_t) * (size_t)B * W, cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess && rc == HOBO_OK && o.ev_end) e = cudaEventRecord((cudaEvent_t)o.ev_end, st);
    if (e == cudaSuccess && rc == HOBO_OK) e = launch_energy_fp64(h, bestX, B, bestE, st);
    if (e == cudaSuccess && rc == HOBO_OK && record && nrec > 0) {
        record_labels_kernel<<<(unsigned)((nrec + 255) / 256), 256, 0, st>>>(rx, bestX, nrec, rec_states, N, W, o.rec_y);
        e = cudaGetLastError();
    }
    void* fr[] = {d_beta, ownX ? d_X : nullptr, ownE ? d_E : nullptr, d_g, d_bE, tables, tf, rx};
    for (void* p : fr)
        if (p) cudaFreeAsync(p, st);
    if (rc != HOBO_OK) return rc;
    if (e != cudaSuccess) return mfail(HOBO_ERR_CUDA, std::string("learned anneal: ") + cudaGetErrorString(e));
    set_error("");
    return HOBO_OK;
}

extern "C" int hobo_mlp_score_tables(hobo_mlp_h m, const float* beta, int S, int G, float vmax, float* tables,
                                     void* stream)
{
    using namespace hobo;
    if (!m) return mfail(HOBO_ERR_ARG, "NULL network");
    if (S < 0) return mfail(HOBO_ERR_ARG, "negative S");
    if (G < 2 || G > (1 << 16)) return mfail(HOBO_ERR_ARG, "G must be 2..65536");
    if (!(vmax > 0.f) || !std::isfinite(vmax)) return mfail(HOBO_ERR_ARG, "vmax must be finite and > 0");
    if (S == 0) return HOBO_OK;
    if (!beta || !tables) return mfail(HOBO_ERR_ARG, "NULL beta or tables");
    cudaStream_t st = (cudaStream_t)stream;
    float* tf = nullptr;
    cudaError_t e = cudaSuccess;
    if (!m->use_tc) e = cudaMallocAsync((void**)&tf, sizeof(float) * (size_t)S * 2 * G * 3, st);
    if (e == cudaSuccess) e = mlp_tables(m, beta, S, G, vmax, tables, tf, m->status, st);
    if (tf) cudaFreeAsync(tf, st);
    if (e != cudaSuccess) return mfail(HOBO_ERR_CUDA, std::string("mlp score tables: ") + cudaGetErrorString(e));
    return HOBO_OK;
}
