// Host side of the C ABI: argument validation, canonicalisation of the HOBO
// tensor into folded monomials, construction of the device layouts, and the
// launch sequences of hobo_energy / hobo_anneal.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda_bf16.h>
#include "hobo_internal.h"

namespace hobo {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

static int fail(int code, const std::string& msg)
{
    set_error(msg);
    return code;
}

static int cuda_fail(cudaError_t e, const char* where)
{
    return fail(HOBO_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define HOBO_CUDA(call)                                                  \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);              \
    } while (0)

// A folded monomial: its distinct variables (ascending) and coefficient.
struct Mono {
    uint16_t v[HOBO_MAX_ORDER];
    uint8_t d;
};

static bool mono_less(const Mono& a, const Mono& b)
{
    if (a.d != b.d) return a.d < b.d;
    for (int q = 0; q < a.d; ++q)
        if (a.v[q] != b.v[q]) return a.v[q] < b.v[q];
    return false;
}

static bool mono_eq(const Mono& a, const Mono& b)
{
    if (a.d != b.d) return false;
    for (int q = 0; q < a.d; ++q)
        if (a.v[q] != b.v[q]) return false;
    return true;
}

struct Entry {
    Mono m;
    double c;
};

// Fold one tensor entry: sort its indices and drop repeats (x*x = x).
static bool fold_entry(const int64_t* tup, int order, int N, Mono& m)
{
    int64_t s[HOBO_MAX_ORDER];
    for (int q = 0; q < order; ++q) {
        if (tup[q] < 0 || tup[q] >= N) return false;
        s[q] = tup[q];
    }
    std::sort(s, s + order);
    int d = 0;
    for (int q = 0; q < order; ++q)
        if (q == 0 || s[q] != s[q - 1]) m.v[d++] = (uint16_t)s[q];
    for (int q = d; q < HOBO_MAX_ORDER; ++q) m.v[q] = 0;
    m.d = (uint8_t)d;
    return true;
}

template <typename T>
static int upload(T** dst, const std::vector<T>& src)
{
    *dst = nullptr;
    if (src.empty()) return HOBO_OK;
    cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * src.size());
    if (e != cudaSuccess) return fail(HOBO_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    e = cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    return HOBO_OK;
}

static void free_layouts(DevLayouts& d)
{
    void* ptrs[] = {d.tvars, d.tfix, d.fptr, d.fvars, d.ffix, d.cptr, d.chdr,
                    d.ltgt, d.lcnt, d.ucoef, d.uconds, d.uent, d.a, d.S2, d.S3, d.S3col, d.S3bf, d.S3limb, d.rs_a, d.rs_S2,
                    d.C3fix, d.S2fix, d.afix, d.pair_m, d.pair_j, d.S4bf, d.S3flimb, d.fa, d.SKbf, d.kmask, d.kmin};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    d = DevLayouts{};
}

static uint16_t bf16_bits_rn(float f)
{
    __nv_bfloat16 b = __float2bfloat16_rn(f);
    uint16_t u;
    std::memcpy(&u, &b, 2);
    return u;
}

static float bf16_value(uint16_t u)
{
    uint32_t w = (uint32_t)u << 16;
    float f;
    std::memcpy(&f, &w, 4);
    return f;
}

static double choose_split(double c, int nsplit, uint16_t out[3])
{
    double r = c;
    for (int q = 0; q < nsplit; ++q) {
        out[q] = bf16_bits_rn((float)r);
        r -= (double)bf16_value(out[q]);
    }
    return r;   // residual not represented
}

// bf16 bits of a small integer (|v| <= 256: exact in bf16)
static uint16_t bf16_of_small_int(int v)
{
    const float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

// Limb planes of the fixed-point cubic coefficients for the exact
// tensor-core re-score (layout in DevLayouts).  Left out (the CUDA-core
// re-score stays in use) when a partial sum could leave 62 bits.
static int build_exact_limbs(hobo_instance* h, const std::vector<Entry>& mono)
{
    DevLayouts& d = h->d;
    const int N = h->N;
    const int S = h->integer ? 0 : d.fix_shift;
    long long maxC = 0;
    double sumC = 0.0;
    for (auto& e : mono) {
        const long long f = std::llrint(std::ldexp(e.c, S));
        maxC = std::max(maxC, f < 0 ? -f : f);
        sumC += std::fabs((double)f);
    }
    if (sumC >= 4.0e18 || (double)maxC * N * N >= 4.0e18) return HOBO_OK;
    int L = 1;
    while (L < 8 && maxC >= (1LL << (8 * L - 1))) ++L;
    const size_t plane = (size_t)N * d.NJ * d.KP;
    std::vector<uint16_t> limbs(plane * L, 0);
    std::vector<long long> ra((size_t)N, 0), rs2((size_t)N * N, 0);
    for (auto& e : mono) {
        const long long f = std::llrint(std::ldexp(e.c, S));
        if (e.m.d == 1) ra[e.m.v[0]] = f;
        else if (e.m.d == 2) rs2[(size_t)e.m.v[0] * N + e.m.v[1]] = f;
        else {
            const uint64_t u = (uint64_t)f;
            const size_t at = ((size_t)e.m.v[0] * d.NJ + e.m.v[1]) * d.KP + e.m.v[2];
            for (int q = 0; q < L; ++q) {
                int limb = (int)((u >> (8 * q)) & 0xFFu);
                if (q == L - 1 && limb >= 128) limb -= 256;     // signed top limb
                limbs[q * plane + at] = bf16_of_small_int(limb);
            }
        }
    }
    int rc;
    if ((rc = upload(&d.S3limb, limbs)) || (rc = upload(&d.rs_a, ra)) || (rc = upload(&d.rs_S2, rs2))) return rc;
    d.rs_L = L;
    d.rs_shift = S;
    if (make_tc_tensor_map_rs(h) != cudaSuccess) {
        (void)cudaGetLastError();
        d.tmap_rs_ok = false;
    }
    return HOBO_OK;
}

// Limb planes of the fixed-point coefficients for the exact energy/field
// contraction on the tensor cores (layout in DevLayouts): each cubic
// monomial {v0 < v1 < v2} goes to the slab of each of its members m, at row
// j and column l > j of the other two; each pair {m, j} to the diagonal
// (j, j) of m's slab and (m, m) of j's.  The scale keeps the sum of all |C|
// below 2^62, so every field and energy sum fits in 64 bits and at most 8
// limbs are needed.
static int build_field_limbs(hobo_instance* h, const std::vector<Entry>& mono)
{
    DevLayouts& d = h->d;
    const int N = h->N;
    const int S = h->integer ? 0 : d.fix_shift;
    long long maxC = 0;
    for (auto& e : mono) {
        const long long f = std::llrint(std::ldexp(e.c, S));
        if (e.m.d >= 2) maxC = std::max(maxC, f < 0 ? -f : f);
    }
    int L = 1;
    while (L < 8 && maxC >= (1LL << (8 * L - 1))) ++L;
    const int KP = d.KP;
    const size_t plane = (size_t)N * KP * KP;
    std::vector<uint16_t> limbs(plane * L, 0);
    std::vector<long long> fa((size_t)N, 0);
    auto put = [&](size_t at, long long f) {
        const uint64_t u = (uint64_t)f;
        for (int q = 0; q < L; ++q) {
            int limb = (int)((u >> (8 * q)) & 0xFFu);
            if (q == L - 1 && limb >= 128) limb -= 256;     // signed top limb
            limbs[q * plane + at] = bf16_of_small_int(limb);
        }
    };
    for (auto& e : mono) {
        const long long f = std::llrint(std::ldexp(e.c, S));
        if (e.m.d == 1) {
            fa[e.m.v[0]] = f;
        } else if (e.m.d == 2) {
            const int m = e.m.v[0], j = e.m.v[1];
            put(((size_t)m * KP + j) * KP + j, f);
            put(((size_t)j * KP + m) * KP + m, f);
        } else {
            const int v[3] = {e.m.v[0], e.m.v[1], e.m.v[2]};
            // (m, j, l): each member as m, the other two ascending
            const int at3[3][3] = {{v[0], v[1], v[2]}, {v[1], v[0], v[2]}, {v[2], v[0], v[1]}};
            for (auto& t : at3) put(((size_t)t[0] * KP + t[1]) * KP + t[2], f);
        }
    }
    int rc;
    if ((rc = upload(&d.S3flimb, limbs)) || (rc = upload(&d.fa, fa))) return rc;
    d.fl_L = L;
    d.fl_shift = S;
    if (make_tc_tensor_map_fl(h) != cudaSuccess) {
        (void)cudaGetLastError();
        d.tmap_fl_ok = false;
    }
    return HOBO_OK;
}

static int build_instance(hobo_instance* h, std::vector<Entry>& mono, unsigned flags);

static void destroy_instance(hobo_instance* h)
{
    if (!h) return;
    destroy_instance(h->low);
    free_layouts(h->d);
    if (h->status && h->owns_status) cudaFree(h->status);
    delete h;
}

// Order-4 tensor-core layout: the quartic part as split bf16 planes of the
// symmetric tensor (every permutation of a monomial's four indices holds
// its coefficient), the lower degrees as a child instance on the term-list
// path.  Left out (term-list path for everything) if the planes cannot be
// described to TMA.
static int build_tc4(hobo_instance* h, const std::vector<Entry>& mono, unsigned flags, double maxabs)
{
    DevLayouts& d = h->d;
    const int N = h->N;
    std::vector<Entry> lower;
    for (auto& e : mono)
        if (e.m.d < 4) lower.push_back(e);
    if (!lower.empty()) {
        hobo_instance* lo = new (std::nothrow) hobo_instance();
        if (!lo) return fail(HOBO_ERR_OOM, "host allocation failed");
        lo->N = N;
        lo->order = 3;
        lo->device = h->device;
        lo->num_sms = h->num_sms;
        lo->status = h->status;
        lo->owns_status = false;
        const int rc = build_instance(lo, lower, HOBO_FORCE_SPARSE);
        if (rc != HOBO_OK) { destroy_instance(lo); return rc; }
        h->low = lo;
    }
    int nsplit = 3;
    if (h->integer && maxabs < 65536.0 && !(flags & HOBO_SPLIT3)) nsplit = 2;
    if (!h->integer && (flags & HOBO_SPLIT2)) nsplit = 2;
    const int N4 = (N + 3) & ~3;
    d.nsplit4 = nsplit;
    d.R4 = N4 * 64;
    const size_t plane = (size_t)N * d.R4 * 64;
    std::vector<uint16_t> planes(plane * nsplit, 0);
    for (auto& e : mono) {
        if (e.m.d != 4) continue;
        uint16_t sp[3];
        choose_split(e.c, nsplit, sp);
        int v[4] = {e.m.v[0], e.m.v[1], e.m.v[2], e.m.v[3]};
        std::sort(v, v + 4);
        do {
            const size_t at = ((size_t)v[0] * d.R4 + (size_t)v[1] * 64 + v[2]) * 64 + v[3];
            for (int q = 0; q < nsplit; ++q) planes[q * plane + at] = sp[q];
        } while (std::next_permutation(v, v + 4));
    }
    int rc;
    if ((rc = upload(&d.S4bf, planes))) return rc;
    if (make_tc4_tensor_map(h) != cudaSuccess) {
        (void)cudaGetLastError();
        d.tmap4_ok = false;
    }
    return HOBO_OK;
}

// Order-5/6 tensor-core layout (layout in DevLayouts): rows over the sorted
// (k-2)-subsets of the variables in lexicographic order, each top-degree
// monomial placed once per member m at row (m, its other members but the
// largest), column = that largest member; degrees < k in a child instance
// (which may take a tensor-core path of its own).  Left out (term-list path
// for everything) beyond 2 GB of planes or if the planes cannot be
// described to TMA.
static int build_tck(hobo_instance* h, const std::vector<Entry>& mono, unsigned flags, double maxabs)
{
    DevLayouts& d = h->d;
    const int N = h->N, k = h->order, pk = k - 2;
    // sorted pk-subsets in lexicographic order, by prefix bit mask
    std::vector<unsigned long long> masks;
    std::vector<uint8_t> mins;
    {
        std::vector<int> c(pk);
        for (int q = 0; q < pk; ++q) c[q] = q;
        while (pk <= N) {
            unsigned long long mk = 0;
            for (int q = 0; q < pk; ++q) mk |= 1ull << c[q];
            masks.push_back(mk);
            mins.push_back((uint8_t)c[0]);
            int q = pk - 1;
            while (q >= 0 && c[q] == N - pk + q) --q;
            if (q < 0) break;
            ++c[q];
            for (int r = q + 1; r < pk; ++r) c[r] = c[r - 1] + 1;
        }
    }
    const int R = (int)masks.size();
    const int RK = (R + 255) / 256 * 256;
    int nsplit = 3;
    if (h->integer && maxabs < 65536.0 && !(flags & HOBO_SPLIT3)) nsplit = 2;
    if (!h->integer && (flags & HOBO_SPLIT2)) nsplit = 2;
    const size_t plane = (size_t)N * RK * 64;
    if ((double)plane * nsplit * 2.0 > 2.0e9) return HOBO_OK;
    std::vector<Entry> lower;
    for (auto& e : mono)
        if (e.m.d < k) lower.push_back(e);
    if (!lower.empty()) {
        hobo_instance* lo = new (std::nothrow) hobo_instance();
        if (!lo) return fail(HOBO_ERR_OOM, "host allocation failed");
        lo->N = N;
        lo->order = k - 1;
        lo->device = h->device;
        lo->num_sms = h->num_sms;
        lo->status = h->status;
        lo->owns_status = false;
        const int rc = build_instance(lo, lower, flags & (HOBO_SPLIT2 | HOBO_SPLIT3));
        if (rc != HOBO_OK) { destroy_instance(lo); return rc; }
        h->low = lo;
    }
    std::unordered_map<unsigned long long, int> row_of;
    row_of.reserve((size_t)R * 2);
    for (int r = 0; r < R; ++r) row_of[masks[r]] = r;
    std::vector<uint16_t> planes(plane * nsplit, 0);
    for (auto& e : mono) {
        if (e.m.d != k) continue;
        uint16_t sp[3];
        choose_split(e.c, nsplit, sp);
        for (int a = 0; a < k; ++a) {
            const int m = e.m.v[a];
            // the other members, ascending (e.m.v is sorted): prefix + largest
            unsigned long long mk = 0;
            int l = -1, n = 0;
            for (int b = 0; b < k; ++b) {
                if (b == a) continue;
                if (++n == k - 1) l = e.m.v[b];
                else mk |= 1ull << e.m.v[b];
            }
            const size_t at = ((size_t)m * RK + row_of.at(mk)) * 64 + l;
            for (int q = 0; q < nsplit; ++q) planes[q * plane + at] = sp[q];
        }
    }
    masks.resize(RK, 0ull);
    mins.resize(RK, (uint8_t)255);
    d.nsplitK = nsplit;
    d.RK = RK;
    int rc;
    if ((rc = upload(&d.SKbf, planes)) || (rc = upload(&d.kmask, masks)) || (rc = upload(&d.kmin, mins))) return rc;
    if (make_tck_tensor_map(h) != cudaSuccess) {
        (void)cudaGetLastError();
        d.tmapK_ok = false;
    }
    return HOBO_OK;
}

// Build every layout from the folded monomial list (sorted by degree, then
// variables) and upload it.
static int build_instance(hobo_instance* h, std::vector<Entry>& mono, unsigned flags)
{
    const int N = h->N, K = h->order;
    h->KF = std::max(K - 1, 1);
    // condition slots per update entry: the sweep kernels are compiled for
    // 1, 2 or 6 slots, so the layout stride is rounded up to one of those
    h->KU = K <= 3 ? 1 : (K == 4 ? 2 : 6);
    // variable slots per monomial in the monomial list (8- or 16-byte rows)
    h->KS = K <= 4 ? 4 : 8;
    h->W = (N + 31) / 32;

    double abs_sum = 0.0, maxabs = 0.0;
    bool all_int = true;
    for (auto& e : mono) {
        h->terms[e.m.d]++;
        abs_sum += std::fabs(e.c);
        maxabs = std::max(maxabs, std::fabs(e.c));
        if (e.c != std::nearbyint(e.c)) all_int = false;
    }
    h->abs_sum = abs_sum;
    h->integer = all_int && abs_sum < 16777216.0;
    if ((flags & HOBO_INTEGER) && !h->integer)
        return fail(HOBO_ERR_NOT_EXACT, all_int ? "sum of |coefficients| >= 2^24"
                                                : "non-integer coefficient with HOBO_INTEGER");

    const int64_t M = (int64_t)mono.size();
    DevLayouts& d = h->d;
    d.M = M;

    // (1) monomial list
    {
        const int KS = h->KS;
        std::vector<uint16_t> tv((size_t)std::max<int64_t>(M, 1) * KS, (uint16_t)N);
        std::vector<long long> cfix((size_t)std::max<int64_t>(M, 1), 0);
        // fixed-point scale: sum |c| * 2^S < 2^62 keeps every partial sum in range
        int S = 0;
        if (abs_sum > 0.0) {
            int ex;
            std::frexp(abs_sum, &ex);          // abs_sum < 2^ex
            S = 62 - ex;
        }
        d.fix_shift = S;
        for (int64_t t = 0; t < M; ++t) {
            for (int q = 0; q < mono[t].m.d; ++q) tv[(size_t)t * KS + q] = mono[t].m.v[q];
            cfix[t] = std::llrint(std::ldexp(mono[t].c, S));
        }
        int rc;
        if ((rc = upload(&d.tvars, tv)) || (rc = upload(&d.tfix, cfix)))
            return rc;
    }
    // (2) field list by variable
    {
        const int KF = K - 1;
        const int KV = KF <= 2 ? 2 : (KF <= 4 ? 4 : 8);
        d.KV = KV;
        std::vector<int64_t> ptr((size_t)N + 1, 0);
        for (auto& e : mono)
            for (int q = 0; q < e.m.d; ++q) ptr[e.m.v[q] + 1]++;
        for (int j = 0; j < N; ++j) ptr[j + 1] += ptr[j];
        d.F = ptr[N];
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        std::vector<uint16_t> fv((size_t)std::max<int64_t>(d.F, 1) * KV, (uint16_t)N);
        std::vector<long long> fc((size_t)std::max<int64_t>(d.F, 1), 0);
        for (auto& e : mono)
            for (int q = 0; q < e.m.d; ++q) {
                const int j = e.m.v[q];
                const int64_t at = fill[j]++;
                int s = 0;
                for (int r = 0; r < e.m.d; ++r)
                    if (r != q) fv[(size_t)at * KV + s++] = e.m.v[r];
                fc[at] = std::llrint(std::ldexp(e.c, d.fix_shift));
            }
        int rc;
        if ((rc = upload(&d.fptr, ptr)) || (rc = upload(&d.fvars, fv)) || (rc = upload(&d.ffix, fc)))
            return rc;
    }

    // dense layout decision: order 3, N <= 512, cubic part at least 25% full
    const double c3 = (double)N * (N - 1) * (N - 2) / 6.0;
    bool dense = false;
    if (K == 3 && N <= 512 && !(flags & HOBO_FORCE_SPARSE)) {
        if ((flags & HOBO_FORCE_DENSE) || (c3 > 0 && (double)h->terms[3] >= 0.25 * c3)) dense = true;
    }
    h->dense = dense;

    if (dense) {
        const int P = (N + 3) & ~3;
        std::vector<float> a((size_t)N, 0.0f), S2((size_t)N * P, 0.0f);
        std::vector<float> S3((size_t)N * N * P, 0.0f);
        for (auto& e : mono) {
            const float c = (float)e.c;
            if (e.m.d == 1) a[e.m.v[0]] = c;
            else if (e.m.d == 2) {
                const int i = e.m.v[0], j = e.m.v[1];
                S2[(size_t)i * P + j] = c;
                S2[(size_t)j * P + i] = c;
            } else {
                const int v[3] = {e.m.v[0], e.m.v[1], e.m.v[2]};
                const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
                for (auto& pm : perm)
                    S3[((size_t)v[pm[0]] * N + v[pm[1]]) * P + v[pm[2]]] = c;
            }
        }
        {
            // exact fixed-point copies for the structured re-score
            std::vector<long long> c3((size_t)N * N * N, 0), c2((size_t)N * N, 0), c1((size_t)N, 0);
            for (auto& e : mono) {
                const long long f = std::llrint(std::ldexp(e.c, d.fix_shift));
                if (e.m.d == 1) c1[e.m.v[0]] = f;
                else if (e.m.d == 2) c2[(size_t)e.m.v[0] * N + e.m.v[1]] = f;
                else c3[((size_t)e.m.v[0] * N + e.m.v[1]) * N + e.m.v[2]] = f;
            }
            std::vector<uint16_t> pm, pj;
            for (int m = 0; m < N; ++m)
                for (int j = m + 1; j < N; ++j) { pm.push_back((uint16_t)m); pj.push_back((uint16_t)j); }
            if (pm.empty()) { pm.push_back(0); pj.push_back(0); }
            int rc2;
            if ((rc2 = upload(&d.C3fix, c3)) || (rc2 = upload(&d.S2fix, c2)) || (rc2 = upload(&d.afix, c1)) ||
                (rc2 = upload(&d.pair_m, pm)) || (rc2 = upload(&d.pair_j, pj)))
                return rc2;
        }
        std::vector<double> colsum((size_t)N * P, 0.0);
        for (auto& e : mono)
            if (e.m.d == 3) {
                const int v[3] = {e.m.v[0], e.m.v[1], e.m.v[2]};
                // slab i, column j collects c over the third member l
                for (int q = 0; q < 3; ++q)
                    for (int r = 0; r < 3; ++r)
                        if (q != r) colsum[(size_t)v[q] * P + v[r]] += (double)(float)e.c;
            }
        std::vector<float> S3col(colsum.begin(), colsum.end());
        // the sweep's slabs: slab i's N rows, then its ceil(N/2) pair rows,
        // row q the float32 sum of rows 2q and 2q + 1 (the update reads one
        // pair row where both bits of a pair are listed)
        const int NS = N + (N + 1) / 2;
        std::vector<float> S3x((size_t)N * NS * P, 0.0f);
        for (int i = 0; i < N; ++i) {
            const float* src = S3.data() + (size_t)i * N * P;
            float* dst = S3x.data() + (size_t)i * NS * P;
            std::copy(src, src + (size_t)N * P, dst);
            for (int q = 0; 2 * q < N; ++q)
                for (int j = 0; j < P; ++j) {
                    const float r0 = src[(size_t)(2 * q) * P + j];
                    const float r1 = 2 * q + 1 < N ? src[(size_t)(2 * q + 1) * P + j] : 0.0f;
                    dst[(size_t)(N + q) * P + j] = r0 + r1;
                }
        }
        int rc;
        if ((rc = upload(&d.a, a)) || (rc = upload(&d.S2, S2)) || (rc = upload(&d.S3, S3x)) ||
            (rc = upload(&d.S3col, S3col)))
            return rc;

        // bf16 split planes for the tensor-core contraction (N <= 256):
        // [q][m][j][l], rows (m, j) padded to NJ, K = l padded to KP.
        if (N <= 256) {
            // two planes represent integers below 2^16 exactly; float
            // coefficients need three (8+8+8 bits cover float32's 24)
            int nsplit = 3;
            if (h->integer && maxabs < 65536.0 && !(flags & HOBO_SPLIT3)) nsplit = 2;
            if (!h->integer && (flags & HOBO_SPLIT2)) nsplit = 2;
            d.nsplit = nsplit;
            d.NJ = (N + 15) & ~15;
            d.KP = (N + 63) & ~63;
            const size_t plane = (size_t)N * d.NJ * d.KP;
            std::vector<uint16_t> planes(plane * nsplit, 0);
            for (auto& e : mono) {
                if (e.m.d != 3) continue;
                uint16_t sp[3];
                choose_split(e.c, nsplit, sp);
                const int v[3] = {e.m.v[0], e.m.v[1], e.m.v[2]};
                const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
                for (auto& pm : perm)
                    for (int q = 0; q < nsplit; ++q)
                        planes[q * plane + ((size_t)v[pm[0]] * d.NJ + v[pm[1]]) * d.KP + v[pm[2]]] = sp[q];
            }
            if ((rc = upload(&d.S3bf, planes))) return rc;
            if (make_tc_tensor_map(h) != cudaSuccess) {
                (void)cudaGetLastError();
                d.tmap_ok = false;
            }
            if (!(flags & HOBO_RESCORE_CUDA_CORES) && (rc = build_exact_limbs(h, mono))) return rc;
            if ((rc = build_field_limbs(h, mono))) return rc;
        }
    } else {
        // order-4 tensor-core contraction when the quartic part is dense
        if (K == 4 && N <= 64 && !(flags & HOBO_FORCE_SPARSE)) {
            const double c4 = (double)N * (N - 1) * (N - 2) * (N - 3) / 24.0;
            if ((flags & HOBO_FORCE_DENSE) || (c4 > 0 && (double)h->terms[4] >= 0.25 * c4)) {
                const int rc4 = build_tc4(h, mono, flags, maxabs);
                if (rc4 != HOBO_OK) return rc4;
            }
        }
        // order-5/6 tensor-core contraction when the top degree is dense
        if ((K == 5 || K == 6) && N >= K && N <= 64 && !(flags & HOBO_FORCE_SPARSE)) {
            double ck = 1.0;
            for (int q = 0; q < K; ++q) ck = ck * (N - q) / (q + 1);
            if ((flags & HOBO_FORCE_DENSE) || (ck > 0 && (double)h->terms[K] >= 0.25 * ck)) {
                const int rck = build_tck(h, mono, flags, maxabs);
                if (rck != HOBO_OK) return rck;
            }
        }
        // (3) update lists grouped by (flipped bit i, target j)
        const int KU = h->KU;
        std::vector<int32_t> cnt((size_t)N * N, 0);
        int64_t U = 0;
        for (auto& e : mono) {
            if (e.m.d < 2) continue;
            for (int a = 0; a < e.m.d; ++a)
                for (int b = 0; b < e.m.d; ++b)
                    if (a != b) { cnt[(size_t)e.m.v[a] * N + e.m.v[b]]++; ++U; }
        }
        if (U >= (int64_t)INT32_MAX) return fail(HOBO_ERR_UNSUPPORTED, "update list too large");
        std::vector<int32_t> bptr((size_t)N + 1, 0), rtgt, rbeg;
        std::vector<int32_t> cell_rec((size_t)N * N, -1);
        int32_t acc = 0;
        for (int i = 0; i < N; ++i) {
            bptr[i] = (int32_t)rtgt.size();
            for (int j = 0; j < N; ++j) {
                const int32_t c = cnt[(size_t)i * N + j];
                if (!c) continue;
                cell_rec[(size_t)i * N + j] = (int32_t)rtgt.size();
                rtgt.push_back(j);
                rbeg.push_back(acc);
                acc += c;
            }
        }
        bptr[N] = (int32_t)rtgt.size();
        rbeg.push_back(acc);
        std::vector<int32_t> fill(rbeg.begin(), rbeg.end() - 1);
        std::vector<float> uc((size_t)std::max<int64_t>(U, 1), 0.0f);
        std::vector<uint16_t> ucond((size_t)std::max<int64_t>(U, 1) * KU, (uint16_t)N);
        for (auto& e : mono) {
            if (e.m.d < 2) continue;
            for (int a = 0; a < e.m.d; ++a)
                for (int b = 0; b < e.m.d; ++b) {
                    if (a == b) continue;
                    const int32_t rec = cell_rec[(size_t)e.m.v[a] * N + e.m.v[b]];
                    const int32_t at = fill[rec]++;
                    uc[at] = (float)e.c;
                    int s = 0;
                    for (int r = 0; r < e.m.d; ++r)
                        if (r != a && r != b) ucond[(size_t)at * KU + s++] = e.m.v[r];
                }
        }
        d.R = (int64_t)rtgt.size();
        d.U = U;
        // Sliced ELL: the target records of bit i in chunks of 32 (lane =
        // record); entry k of lane l of a chunk at offset + 32 k + l, padded
        // to the chunk's longest record with zero coefficients.
        std::vector<int32_t> cptr((size_t)N + 1, 0);
        std::vector<int2> chdr;
        std::vector<uint16_t> ltgt, lcnt;
        std::vector<float> ec;
        std::vector<uint16_t> econd;
        int64_t eoff = 0;
        for (int i = 0; i < N; ++i) {
            cptr[i] = (int32_t)chdr.size();
            for (int r0 = bptr[i]; r0 < bptr[i + 1]; r0 += 32) {
                const int nrec = std::min(32, bptr[i + 1] - r0);
                int K = 0;
                for (int l = 0; l < nrec; ++l) K = std::max(K, rbeg[r0 + l + 1] - rbeg[r0 + l]);
                chdr.push_back(make_int2((int)eoff, K * 64 + nrec));
                for (int l = 0; l < 32; ++l) {
                    ltgt.push_back(l < nrec ? (uint16_t)rtgt[r0 + l] : (uint16_t)0);
                    lcnt.push_back(l < nrec ? (uint16_t)(rbeg[r0 + l + 1] - rbeg[r0 + l]) : (uint16_t)0);
                }
                ec.resize((size_t)(eoff + 32LL * K), 0.0f);
                econd.resize((size_t)(eoff + 32LL * K) * KU, (uint16_t)N);
                for (int l = 0; l < nrec; ++l)
                    for (int k = 0; k < rbeg[r0 + l + 1] - rbeg[r0 + l]; ++k) {
                        const int64_t src = rbeg[r0 + l] + k, dst = eoff + 32LL * k + l;
                        ec[dst] = uc[src];
                        for (int q = 0; q < KU; ++q) econd[dst * KU + q] = ucond[src * KU + q];
                    }
                eoff += 32LL * K;
                if (eoff >= (int64_t)INT32_MAX) return fail(HOBO_ERR_UNSUPPORTED, "update list too large");
            }
        }
        cptr[N] = (int32_t)chdr.size();
        if (chdr.empty()) { chdr.push_back(make_int2(0, 0)); ltgt.assign(32, 0); lcnt.assign(32, 0); }
        if (ec.empty()) { ec.push_back(0.0f); econd.assign(KU, (uint16_t)N); }
        d.C = (int64_t)chdr.size();
        d.Epad = eoff;
        int rc;
        if ((rc = upload(&d.cptr, cptr)) || (rc = upload(&d.chdr, chdr)) || (rc = upload(&d.ltgt, ltgt)) ||
            (rc = upload(&d.lcnt, lcnt)) || (rc = upload(&d.ucoef, ec)) || (rc = upload(&d.uconds, econd)))
            return rc;
        // packed copy: coefficient bits and up to 2 (or 6) 16-bit conditions
        {
            const size_t ne = ec.size();
            const int words = KU <= 2 ? 2 : 4;
            std::vector<uint32_t> pk(ne * words, 0u);
            for (size_t e = 0; e < ne; ++e) {
                uint32_t cb;
                std::memcpy(&cb, &ec[e], 4);
                pk[e * words] = cb;
                for (int q = 0; q < KU; ++q)
                    pk[e * words + 1 + q / 2] |= (uint32_t)econd[e * KU + q] << (16 * (q & 1));
                for (int q = KU; q < 2 * (words - 1); ++q)   // unused slots: the sentinel N
                    pk[e * words + 1 + q / 2] |= (uint32_t)N << (16 * (q & 1));
            }
            uint32_t* dp = nullptr;
            if ((rc = upload(&dp, pk))) return rc;
            d.uent = dp;
        }
    }
    return HOBO_OK;
}

static int create_from_entries(hobo_h* out, std::vector<Entry>& ent, int order, int N, unsigned flags)
{
    std::stable_sort(ent.begin(), ent.end(), [](const Entry& a, const Entry& b) { return mono_less(a.m, b.m); });
    std::vector<Entry> mono;
    mono.reserve(ent.size());
    for (size_t q = 0; q < ent.size();) {
        size_t r = q;
        double c = 0.0;
        while (r < ent.size() && mono_eq(ent[r].m, ent[q].m)) c += ent[r++].c;
        if (c != 0.0) mono.push_back({ent[q].m, c});
        q = r;
    }
    ent.clear();
    ent.shrink_to_fit();

    if (flags & HOBO_INTEGER) {
        double abs_sum = 0.0;
        bool all_int = true;
        for (auto& e : mono) {
            abs_sum += std::fabs(e.c);
            if (e.c != std::nearbyint(e.c)) all_int = false;
        }
        if (!all_int) return fail(HOBO_ERR_NOT_EXACT, "non-integer coefficient with HOBO_INTEGER");
        if (!(abs_sum < 16777216.0)) return fail(HOBO_ERR_NOT_EXACT, "sum of |coefficients| >= 2^24");
    }
    hobo_instance* h = new (std::nothrow) hobo_instance();
    if (!h) return fail(HOBO_ERR_OOM, "host allocation failed");
    h->N = N;
    h->order = order;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDevice"); }
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaDeviceGetAttribute"); }
    e = cudaMalloc((void**)&h->status, sizeof(int));
    if (e != cudaSuccess) { delete h; return fail(HOBO_ERR_OOM, "cudaMalloc status"); }
    e = cudaMemset(h->status, 0, sizeof(int));
    if (e != cudaSuccess) { cudaFree(h->status); delete h; return cuda_fail(e, "cudaMemset"); }
    const int rc = build_instance(h, mono, flags);
    if (rc != HOBO_OK) {
        const std::string msg = g_err;
        destroy_instance(h);
        set_error(msg);
        return rc;
    }
    *out = h;
    set_error("");
    return HOBO_OK;
}

static int check_shape(int order, int N)
{
    if (order < 1 || order > HOBO_MAX_ORDER) return fail(HOBO_ERR_ORDER, "order must be 1..8");
    if (N < 1 || N > HOBO_MAX_N) return fail(HOBO_ERR_ARG, "N must be 1..1024");
    return HOBO_OK;
}

}  // namespace hobo

using namespace hobo;

int hobo::energy_dispatch(const hobo_instance* h, const uint32_t* X, int B, float* E, float* g, bool flip,
                          int path, cudaStream_t st)
{
    if ((path == 2 || path == 0) && tc4_supported(h)) {
        cudaError_t e = launch_energy_tc4(h, X, B, E, g, flip, st);
        if (e == cudaSuccess) return HOBO_OK;
        return cuda_fail(e, "order-4 tensor-core contraction");
    }
    if ((path == 2 || path == 0) && tck_supported(h)) {
        cudaError_t e = launch_energy_tck(h, X, B, E, g, flip, st);
        if (e == cudaSuccess) return HOBO_OK;
        return cuda_fail(e, "order-5/6 tensor-core contraction");
    }
    if (path == 3) {
        cudaError_t e = launch_energy_tc(h, X, B, E, g, flip, st);
        if (e == cudaSuccess) return HOBO_OK;
        if (e != cudaErrorNotSupported) return cuda_fail(e, "tensor-core contraction");
        (void)cudaGetLastError();
        return fail(HOBO_ERR_UNSUPPORTED, "float32-accumulating tensor-core path needs a dense order-3 instance");
    }
    if (path == 2 || (path == 0 && h->dense)) {
        // exact fixed point on the tensor cores: energies only from the
        // re-score planes, energies and fields from the field planes; the
        // float32-accumulating kernel where neither exists
        cudaError_t e = !g ? launch_energy_exact_f32(h, X, B, E, st) : launch_energy_tc_fix(h, X, B, E, g, flip, st);
        if (e == cudaErrorNotSupported) {
            (void)cudaGetLastError();
            e = launch_energy_tc_fix(h, X, B, E, g, flip, st);
        }
        if (e == cudaErrorNotSupported) {
            (void)cudaGetLastError();
            e = launch_energy_tc(h, X, B, E, g, flip, st);
        }
        if (e == cudaSuccess) return HOBO_OK;
        if (e != cudaErrorNotSupported) return cuda_fail(e, "tensor-core contraction");
        if (path == 2)
            return fail(HOBO_ERR_UNSUPPORTED, "tensor-core path needs a dense order-3 or order-4 instance");
        (void)cudaGetLastError();
    }
    cudaError_t e = launch_energy_terms(h, X, B, E, g, flip, st);
    if (e != cudaSuccess) return cuda_fail(e, "term-list contraction");
    return HOBO_OK;
}

extern "C" {

static int hobo_create_impl(hobo_h* out, const float* T, int order, int N, unsigned flags)
{
    if (!out) return fail(HOBO_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!T) return fail(HOBO_ERR_ARG, "T is NULL");
    int rc = check_shape(order, N);
    if (rc) return rc;
    double total = std::pow((double)N, (double)order);
    if (total > 9.0e15) return fail(HOBO_ERR_ARG, "N^order too large");
    const int64_t n = (int64_t)total;
    std::vector<Entry> ent;
    int64_t tup[HOBO_MAX_ORDER] = {0};
    for (int64_t f = 0; f < n; ++f) {
        if (f > 0) {   // odometer over the index tuple, last index fastest
            for (int q = order - 1; q >= 0; --q) {
                if (++tup[q] < N) break;
                tup[q] = 0;
            }
        }
        const float v = T[f];
        if (v == 0.0f) continue;
        if (!std::isfinite(v)) return fail(HOBO_ERR_ARG, "non-finite tensor entry");
        Entry e;
        fold_entry(tup, order, N, e.m);
        e.c = (double)v;
        ent.push_back(e);
    }
    return create_from_entries(out, ent, order, N, flags);
}

int hobo_create(hobo_h* out, const float* T, int order, int N, unsigned flags)
{
    return hobo::guarded("hobo_create", [&] { return hobo_create_impl(out, T, order, N, flags); });
}

static int hobo_create_terms_impl(hobo_h* out, const int32_t* idx, const float* coef, int64_t nnz, int order,
                                  int N, unsigned flags)
{
    if (!out) return fail(HOBO_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_shape(order, N);
    if (rc) return rc;
    if (nnz < 0 || (nnz > 0 && (!idx || !coef))) return fail(HOBO_ERR_ARG, "bad term arrays");
    std::vector<Entry> ent;
    ent.reserve((size_t)nnz);
    int64_t tup[HOBO_MAX_ORDER];
    for (int64_t t = 0; t < nnz; ++t) {
        for (int q = 0; q < order; ++q) tup[q] = idx[t * order + q];
        const float v = coef[t];
        if (!std::isfinite(v)) return fail(HOBO_ERR_ARG, "non-finite coefficient");
        if (v == 0.0f) continue;
        Entry e;
        if (!fold_entry(tup, order, N, e.m))
            return fail(HOBO_ERR_ARG, "index out of range in term " + std::to_string(t));
        e.c = (double)v;
        ent.push_back(e);
    }
    return create_from_entries(out, ent, order, N, flags);
}

int hobo_create_terms(hobo_h* out, const int32_t* idx, const float* coef, int64_t nnz, int order,
                      int N, unsigned flags)
{
    return hobo::guarded("hobo_create_terms", [&] { return hobo_create_terms_impl(out, idx, coef, nnz, order, N, flags); });
}

void hobo_destroy(hobo_h h)
{
    destroy_instance(h);
}

int hobo_check(hobo_h h, void* stream)
{
    if (!h) return fail(HOBO_ERR_ARG, "NULL instance");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int v = 0;
    e = cudaMemcpy(&v, h->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (v != 0) {
        const int zero = 0;
        cudaMemcpy(h->status, &zero, sizeof(int), cudaMemcpyHostToDevice);
        return fail(HOBO_ERR_TIMEOUT, "a device-side wait gave up (status " + std::to_string(v) + ")");
    }
    return HOBO_OK;
}

int hobo_selftest_timeout(hobo_h h, uint64_t limit_ns, void* stream)
{
    if (!h) return fail(HOBO_ERR_ARG, "NULL instance");
    if (limit_ns == 0 || limit_ns > 1000000000ull) return fail(HOBO_ERR_ARG, "limit_ns must be 1..1e9");
    cudaError_t e = launch_wait_timeout_selftest(h, limit_ns, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "timeout self-test");
    return HOBO_OK;
}

int hobo_info(hobo_h h, hobo_info_t* info)
{
    if (!h || !info) return fail(HOBO_ERR_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->N = h->N;
    info->order = h->order;
    info->words = h->W;
    info->dense = h->dense ? 1 : 0;
    info->integer = h->integer ? 1 : 0;
    for (int q = 0; q <= HOBO_MAX_ORDER; ++q) info->terms[q] = h->terms[q];
    info->abs_sum = h->abs_sum;
    info->tc_limbs = h->d.S3flimb ? h->d.fl_L : 0;
    return HOBO_OK;
}

int hobo_energy_path(hobo_h h, const uint32_t* X, int B, float* E, float* dE, int path, void* stream)
{
    if (!h) return fail(HOBO_ERR_ARG, "NULL instance");
    if (B < 0 || (B > 0 && (!X || !E))) return fail(HOBO_ERR_ARG, "bad X/E/B");
    if (path < 0 || path > 3) return fail(HOBO_ERR_ARG, "path must be 0, 1, 2 or 3");
    if (B == 0) return HOBO_OK;
    return hobo::energy_dispatch(h, X, B, E, dE, true, path, (cudaStream_t)stream);
}

int hobo_energy(hobo_h h, const uint32_t* X, int B, float* E, float* dE, void* stream)
{
    return hobo_energy_path(h, X, B, E, dE, 0, stream);
}

int hobo_energy_fp64(hobo_h h, const uint32_t* X, int B, double* E, void* stream)
{
    if (!h) return fail(HOBO_ERR_ARG, "NULL instance");
    if (B < 0 || (B > 0 && (!X || !E))) return fail(HOBO_ERR_ARG, "bad X/E/B");
    if (B == 0) return HOBO_OK;
    cudaError_t e = launch_energy_fp64(h, X, B, E, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fp64 energy");
    return HOBO_OK;
}

int hobo_anneal(hobo_h h, uint64_t seed, int B, const float* beta, int sweeps, uint32_t* bestX,
                double* bestE, const hobo_anneal_opts* opts, void* stream)
{
    if (!h) return fail(HOBO_ERR_ARG, "NULL instance");
    if (B < 0 || sweeps < 0) return fail(HOBO_ERR_ARG, "negative B or sweeps");
    if (B == 0) return HOBO_OK;
    if (!bestX || !bestE) return fail(HOBO_ERR_ARG, "NULL bestX/bestE");
    if (sweeps > 0 && !beta) return fail(HOBO_ERR_ARG, "NULL beta");
    hobo_anneal_opts o{};
    if (opts) o = *opts;
    if (o.mode != HOBO_ANNEAL_TUNED && o.mode != HOBO_ANNEAL_PLAIN) return fail(HOBO_ERR_ARG, "bad mode");
    if (o.resume && (!o.X_io || !o.bestE32_io)) return fail(HOBO_ERR_ARG, "resume needs X_io and bestE32_io");
    if (o.sweep0 < 0) return fail(HOBO_ERR_ARG, "negative sweep0");
    for (int s = 0; s < sweeps; ++s)
        if (!(beta[s] >= 0.0f) || !std::isfinite(beta[s])) return fail(HOBO_ERR_ARG, "beta must be finite and >= 0");

    cudaStream_t st = (cudaStream_t)stream;
    const int N = h->N, W = h->W;
    float* d_beta = nullptr;
    uint32_t* d_X = o.X_io;
    float* d_g = nullptr;
    float* d_E = nullptr;
    float* d_bE = o.bestE32_io;
    bool own_X = false, own_bE = false;
    int rc = HOBO_OK;
    auto cleanup = [&]() {
        if (d_beta) cudaFreeAsync(d_beta, st);
        if (own_X && d_X) cudaFreeAsync(d_X, st);
        if (d_g && d_g != o.g_io) cudaFreeAsync(d_g, st);
        if (d_E && d_E != o.E_io) cudaFreeAsync(d_E, st);
        if (own_bE && d_bE) cudaFreeAsync(d_bE, st);
    };
#define ACHECK(call, what)                                            \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) { rc = cuda_fail(e_, what); cleanup(); return rc; } \
    } while (0)

    if (sweeps > 0) {
        ACHECK(cudaMallocAsync((void**)&d_beta, sizeof(float) * sweeps, st), "cudaMallocAsync beta");
        ACHECK(cudaMemcpyAsync(d_beta, beta, sizeof(float) * sweeps, cudaMemcpyHostToDevice, st), "beta copy");
    }
    if (!d_X) {
        ACHECK(cudaMallocAsync((void**)&d_X, sizeof(uint32_t) * (size_t)B * W, st), "cudaMallocAsync X");
        own_X = true;
    }
    if (!d_bE) {
        ACHECK(cudaMallocAsync((void**)&d_bE, sizeof(float) * (size_t)B, st), "cudaMallocAsync bestE");
        own_bE = true;
    }
    if (o.g_io) d_g = o.g_io;
    else ACHECK(cudaMallocAsync((void**)&d_g, sizeof(float) * (size_t)B * N, st), "cudaMallocAsync g");
    if (o.E_io) d_E = o.E_io;
    else ACHECK(cudaMallocAsync((void**)&d_E, sizeof(float) * (size_t)B, st), "cudaMallocAsync E");

    if (!o.resume) ACHECK(launch_init_states(d_X, B, N, W, seed, st, (uint32_t)o.state0), "init states");
    if (!(o.resume && o.g_io && o.E_io)) {
        rc = hobo::energy_dispatch(h, d_X, B, d_E, d_g, false, 0, st);
        if (rc != HOBO_OK) { cleanup(); return rc; }
    }

    SweepArgs a;
    a.B = B; a.sweeps = sweeps; a.sweep0 = o.sweep0; a.resume = o.resume; a.seed = seed;
    a.state0 = (uint32_t)o.state0;
    a.S = o.states_per_block;
    a.beta = d_beta; a.X = d_X; a.g = d_g; a.E = d_E; a.bestX = bestX; a.bestE = d_bE;
    a.accepts = o.accepts;
    a.coef_bytes = o.coef_bytes;
    a.write_g = o.g_io != nullptr;
    if (sweeps > 0) {
        if (o.ev_sweep_begin) ACHECK(cudaEventRecord((cudaEvent_t)o.ev_sweep_begin, st), "event record");
        if (o.mode == HOBO_ANNEAL_PLAIN) ACHECK(launch_sweep_plain(h, a, st), "plain sweep");
        else ACHECK(launch_sweep_tuned(h, a, st), "tuned sweep");
        if (o.ev_sweep_end) ACHECK(cudaEventRecord((cudaEvent_t)o.ev_sweep_end, st), "event record");
    } else if (!o.resume) {
        ACHECK(cudaMemcpyAsync(bestX, d_X, sizeof(uint32_t) * (size_t)B * W, cudaMemcpyDeviceToDevice, st), "bestX");
        ACHECK(cudaMemcpyAsync(d_bE, d_E, sizeof(float) * (size_t)B, cudaMemcpyDeviceToDevice, st), "bestE");
    }
    ACHECK(launch_energy_fp64(h, bestX, B, bestE, st), "fp64 re-score");
    cleanup();
    set_error("");
    return HOBO_OK;
#undef ACHECK
}

const char* hobo_last_error(void) { return g_err.c_str(); }

const char* hobo_version(void) { return "hobo-gb300 0.1"; }

}  // extern "C"
