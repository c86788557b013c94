// Batched annealing of many instances of uneven size (the tensor batch
// system of Sec. IV.C applied across instances).
//
// A batch plan owns, for every instance t, contiguous blocks of B_t states
// (packed bits, fields, energies, best states) laid end to end, and a
// descriptor per instance.  The sweep of all instances runs as one
// persistent kernel per layout group (dense / sparse with 1, 2 or 6
// condition slots): its warps take (instance, state) items from a queue
// sorted by decreasing cost.  Initial states, the contraction and the
// re-score are launched per instance; the whole sequence is captured once
// in a CUDA graph and replayed.  The launch shape of the persistent kernel
// (warps per CTA, CTAs per SM) is chosen by timing short runs.  Every state
// is annealed exactly as a per-instance hobo_anneal with the same seed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "hobo_internal.h"
#include "hobo_dev.cuh"
#include "sweep_impl.cuh"

namespace hobo {

SweepDev make_dev(const hobo_instance* h, const SweepArgs& a);
cudaError_t launch_energy_fp64_into(const hobo_instance* h, const uint32_t* X, int B, double* E,
                                    unsigned long long* acc, cudaStream_t st);

struct BatchGroup {
    bool dense = false;
    int KU = 1;
    int Nmax = 0, Wmax = 0;
    int i0 = 0, i1 = 0;        // item range in the queue
    int warps = 8, ctas = 0;   // launch shape (ctas = total CTAs)
    int* counter = nullptr;    // device work counter
};

}  // namespace hobo

struct hobo_batch {
    int n = 0;
    std::vector<hobo_h> hs;
    std::vector<int> B;
    std::vector<int64_t> xoff, goff, soff;   // offsets in words / floats / states
    int64_t total = 0, xwords = 0, gfloats = 0;
    int device = 0, num_sms = 0;
    uint32_t* X = nullptr;
    float* g = nullptr;
    float* E = nullptr;
    float* bE32 = nullptr;
    uint32_t* bestX = nullptr;
    double* bestE = nullptr;
    unsigned long long* acc = nullptr;
    float* beta = nullptr;
    int beta_cap = 0;
    hobo::SweepDev* descs = nullptr;
    std::vector<hobo::SweepDev> hdescs;
    int2* items = nullptr;
    int nitems = 0;
    int2* initmap = nullptr;
    int ninit = 0;
    std::vector<hobo::BatchGroup> groups;
    bool tuned = false;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace hobo {

static int bfail(int code, const std::string& msg)
{
    set_error(msg);
    return code;
}

__global__ void batch_init_kernel(const SweepDev* __restrict__ descs, const int2* __restrict__ map)
{
    const int2 bm = map[blockIdx.x];
    const SweepDev& p = descs[bm.x];
    const int64_t tid = (int64_t)bm.y * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)p.B * p.W) return;
    const int b = (int)(tid / p.W), w = (int)(tid % p.W);
    p.X[tid] = init_word(b, w, p.N, p.k0, p.k1);
}

static void free_batch(hobo_batch* bh)
{
    void* ptrs[] = {bh->X, bh->g, bh->E, bh->bE32, bh->bestX, bh->bestE, bh->acc, bh->beta,
                    bh->descs, bh->items, bh->initmap};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& gr : bh->groups)
        if (gr.counter) cudaFree(gr.counter);
    if (bh->exec) cudaGraphExecDestroy(bh->exec);
    if (bh->cap) cudaStreamDestroy(bh->cap);
}

template <typename T>
static cudaError_t dalloc(T** p, size_t n)
{
    return cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(n, 1));
}

static cudaError_t launch_group_sweep(hobo_batch* bh, const BatchGroup& gr, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(gr.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const int2* items = bh->items + gr.i0;
    const int ni = gr.i1 - gr.i0;
    if (gr.dense) return dispatch_batch<true, 1>(bh->descs, items, ni, gr.counter, gr.Nmax, gr.Wmax, gr.warps, gr.ctas, st);
    if (gr.KU == 1) return dispatch_batch<false, 1>(bh->descs, items, ni, gr.counter, gr.Nmax, gr.Wmax, gr.warps, gr.ctas, st);
    if (gr.KU == 2) return dispatch_batch<false, 2>(bh->descs, items, ni, gr.counter, gr.Nmax, gr.Wmax, gr.warps, gr.ctas, st);
    return dispatch_batch<false, 6>(bh->descs, items, ni, gr.counter, gr.Nmax, gr.Wmax, gr.warps, gr.ctas, st);
}

// initial states and their fields and energies, in stream order
static int enqueue_init(hobo_batch* bh, cudaStream_t st)
{
    if (bh->ninit > 0) {
        batch_init_kernel<<<bh->ninit, 256, 0, st>>>(bh->descs, bh->initmap);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, std::string("batch init: ") + cudaGetErrorString(e));
    }
    for (int t = 0; t < bh->n; ++t) {
        const int rc = energy_dispatch(bh->hs[t], bh->X + bh->xoff[t], bh->B[t], bh->E + bh->soff[t],
                                       bh->g + bh->goff[t], false, 0, st);
        if (rc != HOBO_OK) return rc;
    }
    return HOBO_OK;
}

// init, contraction and sweep of the whole batch (everything but the
// re-score), in stream order
static int enqueue_front(hobo_batch* bh, cudaStream_t st)
{
    const int rc = enqueue_init(bh, st);
    if (rc != HOBO_OK) return rc;
    for (auto& gr : bh->groups) {
        cudaError_t e = launch_group_sweep(bh, gr, st);
        if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, std::string("batch sweep: ") + cudaGetErrorString(e));
    }
    return HOBO_OK;
}

static int enqueue_rescore(hobo_batch* bh, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(bh->acc, 0, sizeof(unsigned long long) * (size_t)bh->total, st);
    for (int t = 0; t < bh->n && e == cudaSuccess; ++t)
        e = launch_energy_fp64_into(bh->hs[t], bh->bestX + bh->xoff[t], bh->B[t], bh->bestE + bh->soff[t],
                                    bh->acc + bh->soff[t], st);
    if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, std::string("batch re-score: ") + cudaGetErrorString(e));
    return HOBO_OK;
}

// Fill the descriptors for a run (seeds, schedule, counters) and upload them.
static int upload_descs(hobo_batch* bh, const uint64_t* seeds, int sweeps, int64_t* accepts, cudaStream_t st)
{
    for (int t = 0; t < bh->n; ++t) {
        SweepArgs a;
        a.B = bh->B[t];
        a.sweeps = sweeps;
        a.seed = seeds[t];
        a.beta = bh->beta;
        a.X = bh->X + bh->xoff[t];
        a.g = bh->g + bh->goff[t];
        a.E = bh->E + bh->soff[t];
        a.bestX = bh->bestX + bh->xoff[t];
        a.bestE = bh->bE32 + bh->soff[t];
        a.accepts = accepts ? accepts + bh->soff[t] : nullptr;
        bh->hdescs[t] = make_dev(bh->hs[t], a);
    }
    cudaError_t e = cudaMemcpyAsync(bh->descs, bh->hdescs.data(), sizeof(SweepDev) * bh->n,
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, std::string("descriptor upload: ") + cudaGetErrorString(e));
    // pageable source: make sure the copy has been staged before the host
    // array is refilled by a later call
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, std::string("descriptor upload: ") + cudaGetErrorString(e));
    return HOBO_OK;
}

static int upload_beta(hobo_batch* bh, const float* beta, int sweeps, cudaStream_t st)
{
    if (sweeps > bh->beta_cap) {
        if (bh->beta) cudaFree(bh->beta);
        bh->beta = nullptr;
        if (dalloc(&bh->beta, (size_t)sweeps) != cudaSuccess) return bfail(HOBO_ERR_OOM, "beta buffer");
        bh->beta_cap = sweeps;
        if (bh->exec) { cudaGraphExecDestroy(bh->exec); bh->exec = nullptr; }
    }
    if (sweeps > 0) {
        cudaError_t e = cudaMemcpyAsync(bh->beta, beta, sizeof(float) * sweeps, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, "beta copy");
    }
    return HOBO_OK;
}

// Launch shapes tried by the tuner: warps per CTA x CTAs per SM.
static const int kTuneWarps[] = {4, 8};
static const int kTuneCtasPerSm[] = {2, 4, 6, 8};

static int autotune(hobo_batch* bh, const uint64_t* seeds, const float* beta, int sweeps, cudaStream_t st)
{
    // the probe anneals 32 sweeps whose temperatures are spread evenly over
    // the whole schedule, so that its mix of update-heavy (hot) and
    // attempt-heavy (cold) sweeps resembles the full run's
    const int probe = std::max(1, std::min(sweeps, 32));
    std::vector<float> pb((size_t)probe);
    for (int k = 0; k < probe; ++k)
        pb[k] = beta[probe > 1 ? (int)((int64_t)k * (sweeps - 1) / (probe - 1)) : 0];
    int rc = upload_beta(bh, pb.data(), probe, st);
    if (rc) return rc;
    if ((rc = upload_descs(bh, seeds, probe, nullptr, st))) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (auto& gr : bh->groups) {
        float best_ms = 1e30f;
        int bw = gr.warps, bc = gr.ctas;
        for (int w : kTuneWarps) {
            for (int c : kTuneCtasPerSm) {
                gr.warps = w;
                gr.ctas = c * bh->num_sms;
                // every trial starts from freshly initialised states; the
                // best of two timings counts
                float ms = 1e30f;
                for (int rep = 0; rep < 2 && !rc; ++rep) {
                    if ((rc = enqueue_init(bh, st))) break;
                    cudaEventRecord(e0, st);
                    if (launch_group_sweep(bh, gr, st) != cudaSuccess) { (void)cudaGetLastError(); ms = 1e30f; break; }
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = bfail(HOBO_ERR_CUDA, "autotune"); break; }
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    ms = std::min(ms, t);
                }
                if (rc) break;
                if (ms < best_ms) { best_ms = ms; bw = w; bc = gr.ctas; }
            }
            if (rc) break;
        }
        gr.warps = bw;
        gr.ctas = bc;
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bh->exec) { cudaGraphExecDestroy(bh->exec); bh->exec = nullptr; }
    bh->tuned = rc == HOBO_OK;
    return rc;
}

static int build_graph(hobo_batch* bh)
{
    if (!bh->cap) {
        cudaError_t e = cudaStreamCreateWithFlags(&bh->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, "capture stream");
    }
    cudaError_t e = cudaStreamBeginCapture(bh->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    int rc = enqueue_front(bh, bh->cap);
    if (rc == HOBO_OK) rc = enqueue_rescore(bh, bh->cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(bh->cap, &graph);
    if (rc != HOBO_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&bh->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { bh->exec = nullptr; return bfail(HOBO_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e)); }
    return HOBO_OK;
}

}  // namespace hobo

using namespace hobo;

extern "C" {

static int hobo_batch_create_impl(hobo_batch_h* out, const hobo_h* hs, int n, const int* B)
{
    if (!out) return bfail(HOBO_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n <= 0 || !hs || !B) return bfail(HOBO_ERR_ARG, "need n > 0 instances and their batch sizes");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, "cudaGetDevice");
    for (int t = 0; t < n; ++t) {
        if (!hs[t]) return bfail(HOBO_ERR_ARG, "NULL instance " + std::to_string(t));
        if (B[t] < 0) return bfail(HOBO_ERR_ARG, "negative batch size for instance " + std::to_string(t));
        if (hs[t]->device != dev) return bfail(HOBO_ERR_ARG, "instance " + std::to_string(t) + " lives on another device");
    }
    hobo_batch* bh = new (std::nothrow) hobo_batch();
    if (!bh) return bfail(HOBO_ERR_OOM, "host allocation failed");
    bh->n = n;
    bh->device = dev;
    cudaDeviceGetAttribute(&bh->num_sms, cudaDevAttrMultiProcessorCount, dev);
    bh->hs.assign(hs, hs + n);
    bh->B.assign(B, B + n);
    bh->xoff.resize(n); bh->goff.resize(n); bh->soff.resize(n);
    for (int t = 0; t < n; ++t) {
        bh->xoff[t] = bh->xwords;
        bh->goff[t] = bh->gfloats;
        bh->soff[t] = bh->total;
        bh->xwords += (int64_t)B[t] * hs[t]->W;
        bh->gfloats += (int64_t)B[t] * hs[t]->N;
        bh->total += B[t];
    }
    bh->hdescs.resize(n);
    // work items grouped by layout kind, each group sorted by decreasing cost
    struct Key { bool dense; int KU; };
    std::vector<Key> kinds;
    std::vector<int2> items;
    std::vector<int> order(n);
    for (int t = 0; t < n; ++t) order[t] = t;
    auto cost = [&](int t) {
        const hobo_instance* h = hs[t];
        const double upd = h->dense ? (double)h->N * h->N / 3.0 : (double)h->d.U / std::max(h->N, 1);
        return (double)h->N * (8.0 + upd / 32.0);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    for (int pass = 0; pass < 4; ++pass) {
        const bool dense = pass == 0;
        const int KU = pass <= 1 ? 1 : (pass == 2 ? 2 : 6);
        BatchGroup gr;
        gr.dense = dense;
        gr.KU = KU;
        gr.i0 = (int)items.size();
        for (int t : order) {
            const hobo_instance* h = hs[t];
            if (h->dense != dense || (!dense && h->KU != KU)) continue;
            gr.Nmax = std::max(gr.Nmax, h->N);
            gr.Wmax = std::max(gr.Wmax, h->W);
            for (int b = 0; b < B[t]; ++b) items.push_back(make_int2(t, b));
        }
        gr.i1 = (int)items.size();
        if (gr.i1 > gr.i0) {
            gr.ctas = 4 * bh->num_sms;
            bh->groups.push_back(gr);
        }
    }
    bh->nitems = (int)items.size();
    std::vector<int2> initmap;
    for (int t = 0; t < n; ++t) {
        const int64_t words = (int64_t)B[t] * hs[t]->W;
        for (int64_t k = 0; k < (words + 255) / 256; ++k) initmap.push_back(make_int2(t, (int)k));
    }
    bh->ninit = (int)initmap.size();
    bool ok = dalloc(&bh->X, bh->xwords) == cudaSuccess && dalloc(&bh->g, bh->gfloats) == cudaSuccess &&
              dalloc(&bh->E, bh->total) == cudaSuccess && dalloc(&bh->bE32, bh->total) == cudaSuccess &&
              dalloc(&bh->bestX, bh->xwords) == cudaSuccess && dalloc(&bh->bestE, bh->total) == cudaSuccess &&
              dalloc(&bh->acc, bh->total) == cudaSuccess && dalloc(&bh->descs, n) == cudaSuccess &&
              dalloc(&bh->items, items.size()) == cudaSuccess && dalloc(&bh->initmap, initmap.size()) == cudaSuccess;
    for (auto& gr : bh->groups) ok = ok && dalloc(&gr.counter, 1) == cudaSuccess;
    if (ok && !items.empty())
        ok = cudaMemcpy(bh->items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok && !initmap.empty())
        ok = cudaMemcpy(bh->initmap, initmap.data(), sizeof(int2) * initmap.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        free_batch(bh);
        delete bh;
        return bfail(HOBO_ERR_OOM, "batch buffers");
    }
    *out = bh;
    return HOBO_OK;
}

int hobo_batch_create(hobo_batch_h* out, const hobo_h* hs, int n, const int* B)
{
    return hobo::guarded("hobo_batch_create", [&] { return hobo_batch_create_impl(out, hs, n, B); });
}

void hobo_batch_destroy(hobo_batch_h bh)
{
    if (!bh) return;
    free_batch(bh);
    delete bh;
}

int hobo_batch_layout(hobo_batch_h bh, int64_t* state_offset, int64_t* word_offset)
{
    if (!bh) return bfail(HOBO_ERR_ARG, "NULL batch");
    for (int t = 0; t < bh->n; ++t) {
        if (state_offset) state_offset[t] = bh->soff[t];
        if (word_offset) word_offset[t] = bh->xoff[t];
    }
    return HOBO_OK;
}

static int hobo_batch_anneal_impl(hobo_batch_h bh, const uint64_t* seeds, const float* beta, int sweeps,
                                  uint32_t* bestX, double* bestE, const hobo_batch_opts* opts, void* stream)
{
    if (!bh) return bfail(HOBO_ERR_ARG, "NULL batch");
    if (!seeds || sweeps < 0 || (sweeps > 0 && !beta) || !bestX || !bestE)
        return bfail(HOBO_ERR_ARG, "bad seeds/beta/sweeps/outputs");
    for (int s = 0; s < sweeps; ++s)
        if (!(beta[s] >= 0.0f) || !std::isfinite(beta[s])) return bfail(HOBO_ERR_ARG, "beta must be finite and >= 0");
    hobo_batch_opts o{};
    if (opts) o = *opts;
    cudaStream_t st = (cudaStream_t)stream;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != bh->device) return bfail(HOBO_ERR_ARG, "batch lives on another device");
    int rc;
    if (o.mode == HOBO_BATCH_GRAPH) {
        if (!bh->tuned && !o.no_autotune && sweeps > 0)
            if ((rc = autotune(bh, seeds, beta, sweeps, st))) return rc;
        if (o.warps_per_cta > 0 || o.ctas_per_sm > 0) {
            for (auto& gr : bh->groups) {
                if (o.warps_per_cta > 0) gr.warps = std::min(8, o.warps_per_cta);
                if (o.ctas_per_sm > 0) gr.ctas = o.ctas_per_sm * bh->num_sms;
            }
            if (bh->exec) { cudaGraphExecDestroy(bh->exec); bh->exec = nullptr; }
        }
        if ((rc = upload_beta(bh, beta, std::max(sweeps, 1), st))) return rc;
        if ((rc = upload_descs(bh, seeds, sweeps, o.accepts, st))) return rc;
        if (!bh->exec && (rc = build_graph(bh))) return rc;
        if (o.ev_begin) cudaEventRecord((cudaEvent_t)o.ev_begin, st);
        cudaError_t e = cudaGraphLaunch(bh->exec, st);
        if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
        if (o.ev_end) cudaEventRecord((cudaEvent_t)o.ev_end, st);
    } else if (o.mode == HOBO_BATCH_PER_INSTANCE_TUNED || o.mode == HOBO_BATCH_PER_INSTANCE_PLAIN) {
        // reference forms: one launch sequence per instance
        if ((rc = upload_beta(bh, beta, std::max(sweeps, 1), st))) return rc;
        if (o.ev_begin) cudaEventRecord((cudaEvent_t)o.ev_begin, st);
        for (int t = 0; t < bh->n; ++t) {
            hobo_instance* h = bh->hs[t];
            const int Bt = bh->B[t];
            if (Bt == 0) continue;
            cudaError_t e = launch_init_states(bh->X + bh->xoff[t], Bt, h->N, h->W, seeds[t], st);
            if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, "init");
            if ((rc = energy_dispatch(h, bh->X + bh->xoff[t], Bt, bh->E + bh->soff[t], bh->g + bh->goff[t], false, 0, st)))
                return rc;
            SweepArgs a;
            a.B = Bt; a.sweeps = sweeps; a.seed = seeds[t]; a.beta = bh->beta;
            a.X = bh->X + bh->xoff[t]; a.g = bh->g + bh->goff[t]; a.E = bh->E + bh->soff[t];
            a.bestX = bh->bestX + bh->xoff[t]; a.bestE = bh->bE32 + bh->soff[t];
            a.accepts = o.accepts ? o.accepts + bh->soff[t] : nullptr;
            e = (o.mode == HOBO_BATCH_PER_INSTANCE_PLAIN) ? launch_sweep_plain(h, a, st) : launch_sweep_tuned(h, a, st);
            if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, std::string("sweep: ") + cudaGetErrorString(e));
            e = launch_energy_fp64(h, bh->bestX + bh->xoff[t], Bt, bh->bestE + bh->soff[t], st);
            if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, "re-score");
        }
        if (o.ev_end) cudaEventRecord((cudaEvent_t)o.ev_end, st);
    } else {
        return bfail(HOBO_ERR_ARG, "bad batch mode");
    }
    cudaError_t e = cudaMemcpyAsync(bestX, bh->bestX, sizeof(uint32_t) * (size_t)bh->xwords, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bestE, bh->bestE, sizeof(double) * (size_t)bh->total, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && o.X_out)
        e = cudaMemcpyAsync(o.X_out, bh->X, sizeof(uint32_t) * (size_t)bh->xwords, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && o.E_out)
        e = cudaMemcpyAsync(o.E_out, bh->E, sizeof(float) * (size_t)bh->total, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return bfail(HOBO_ERR_CUDA, "output copy");
    set_error("");
    return HOBO_OK;
}

int hobo_batch_anneal(hobo_batch_h bh, const uint64_t* seeds, const float* beta, int sweeps,
                      uint32_t* bestX, double* bestE, const hobo_batch_opts* opts, void* stream)
{
    return hobo::guarded("hobo_batch_anneal", [&] { return hobo_batch_anneal_impl(bh, seeds, beta, sweeps, bestX, bestE, opts, stream); });
}

int hobo_batch_launch_shape(hobo_batch_h bh, int group, int* warps_per_cta, int* ctas)
{
    if (!bh || group < 0 || group >= (int)bh->groups.size()) return bfail(HOBO_ERR_ARG, "bad batch/group");
    if (warps_per_cta) *warps_per_cta = bh->groups[group].warps;
    if (ctas) *ctas = bh->groups[group].ctas;
    return HOBO_OK;
}

}  // extern "C"
