// Internal declarations shared by the host library and the kernel files.
#pragma once
#include <cstdint>
#include <exception>
#include <new>
#include <string>
#include <cuda_runtime.h>
#include "hobo.h"

namespace hobo {

// Device copies of one instance's layouts.  All arrays are owned by the
// instance and freed by hobo_destroy.
struct DevLayouts {
    // (1) folded monomial list, all degrees, KS (4 or 8) variable slots per
    //     monomial padded with the sentinel index N (whose bit reads as 1).
    //     Coefficients are fixed point: round(c * 2^fix_shift) with
    //     fix_shift chosen so that the sum of all |c| stays below 2^62, so
    //     every partial sum of them is exact in 64-bit integers.
    int64_t M = 0;
    uint16_t* tvars = nullptr;   // [M][KS]
    long long* tfix = nullptr;   // [M]
    int fix_shift = 0;

    // (2) field list by variable: entry e of variable j holds the fixed-
    //     point coefficient of a monomial containing j and its other
    //     members (KV = 2, 4 or 8 >= order-1 slots, sentinel N).
    int64_t F = 0;
    int KV = 2;
    int64_t* fptr = nullptr;     // [N+1]
    uint16_t* fvars = nullptr;   // [F][KV]
    long long* ffix = nullptr;   // [F]

    // (3) update lists by flipped bit (sparse sweep), sliced ELL: the
    //     target records of bit i are chunks cptr[i]..cptr[i+1] of 32 records
    //     (lane = record); chunk c has header chdr[c] = (entry offset,
    //     K * 64 + records), per-lane target ltgt[32c + l] and entry count
    //     lcnt[32c + l]; entry k of lane l sits at offset + 32k + l and holds
    //     a coefficient of a monomial containing i and the target, and the
    //     monomial's other members (KU slots, sentinel N), zero-padded to K.
    int64_t R = 0, U = 0, C = 0, Epad = 0;
    int32_t* cptr = nullptr;     // [N+1]
    int2* chdr = nullptr;        // [C]
    uint16_t* ltgt = nullptr;    // [C][32]
    uint16_t* lcnt = nullptr;    // [C][32]
    float* ucoef = nullptr;      // [Epad]
    uint16_t* uconds = nullptr;  // [Epad][KU]
    // the same entries packed for the tuned sweeps, one load each: KU <= 2:
    // uint2 (coefficient bits, conditions c0 | c1 << 16); KU = 6: uint4
    // (coefficient bits, c0 | c1 << 16, c2 | c3 << 16, c4 | c5 << 16)
    void* uent = nullptr;

    // (4) dense order<=3 layout: linear a[N], symmetric pair matrix S2[N][N]
    //     and symmetric cubic tensor S3[N][N][N] (zero where indices repeat),
    //     float32; bf16 split planes of S3 for the tensor-core contraction.
    float* a = nullptr;
    float* S2 = nullptr;
    float* S3 = nullptr;         // [N][N + ceil(N/2)][P]: slab i's rows, then its pair rows
    float* S3col = nullptr;      // [N][P]: S3col[i][j] = sum_l S3[i][l][j]
    // exact re-score of dense instances: fixed-point coefficients (scale
    // 2^fix_shift) C3fix[m][j][l] for m < j < l (else 0), S2fix[m][j] for
    // m < j, afix[m]; and the list of pairs m < j
    long long* C3fix = nullptr;
    long long* S2fix = nullptr;
    long long* afix = nullptr;
    uint16_t* pair_m = nullptr;
    uint16_t* pair_j = nullptr;
    // bf16 planes [nsplit][N][NJ][KP]: plane q, row (m, j), column l;
    // NJ = N rounded up to 16, KP = N rounded up to 64, zero padded.
    uint16_t* S3bf = nullptr;
    int nsplit = 0, NJ = 0, KP = 0;
    alignas(64) unsigned char tmap[128] = {};   // CUtensorMap of the planes
    bool tmap_ok = false;
    // exact re-score on the tensor cores (N <= 256): the fixed-point cubic
    // coefficients C[m][j][l] = round(c * 2^rs_shift), m < j < l (else 0),
    // as rs_L signed 8-bit limbs (C = sum_q limb_q 2^(8q), limbs below the
    // top unsigned), each limb an exact bf16 plane [rs_L][N][NJ][KP]; linear
    // and pair coefficients at the same scale.  rs_shift = 0 for integer
    // instances, fix_shift otherwise (the same integers as C3fix).
    uint16_t* S3limb = nullptr;
    long long* rs_a = nullptr;    // [N]
    long long* rs_S2 = nullptr;   // [N][N], m < j
    int rs_L = 0, rs_shift = 0;
    alignas(64) unsigned char tmap_rs[128] = {};
    bool tmap_rs_ok = false;
    // exact energies and fields on the tensor cores (N <= 256): the
    // fixed-point coefficients C = round(c * 2^fl_shift) of every monomial
    // containing m in m's slab, a cubic {m, j, l} at row j, column l > j
    // (the upper triangle), a pair {m, j} on the diagonal (j, j) (rows and
    // columns = m hold zeros), as fl_L limbs in exact bf16 planes
    // [fl_L][N][KP][KP] (rows padded to KP = N rounded up to 64); linear
    // coefficients fa[N] at the same scale.  fl_shift = 0 for integer
    // instances, fix_shift otherwise, so results equal the term-list
    // path's.
    uint16_t* S3flimb = nullptr;
    long long* fa = nullptr;
    int fl_L = 0, fl_shift = 0;
    alignas(64) unsigned char tmap_fl[128] = {};
    bool tmap_fl_ok = false;
    // order-4 tensor-core contraction (order-4 instances, N <= 64, quartic
    // part dense): the symmetric quartic tensor as bf16 split planes
    // [nsplit4][N][R4][64], row (j, k) = j * 64 + k (k >= N zero), R4 = (N
    // rounded up to 4) * 64, K = l padded to 64; monomials of degree <= 3
    // go to a child instance on the term-list path.
    uint16_t* S4bf = nullptr;
    int nsplit4 = 0, R4 = 0;
    alignas(64) unsigned char tmap4[128] = {};
    bool tmap4_ok = false;
    // order-5/6 tensor-core contraction (N <= 64, top degree dense): rows
    // (m, P) over the sorted (k-2)-subsets P of the variables in
    // lexicographic order, RK of them padded to 256; plane entry (m, P, l) =
    // coefficient of P + {l} + {m} for l > max P, l and m not in P; bf16
    // split planes [nsplitK][N][RK][64]; kmask [RK] the prefix bits, kmin [RK]
    // the prefix's smallest member; degrees < k in the child instance.
    uint16_t* SKbf = nullptr;
    unsigned long long* kmask = nullptr;
    uint8_t* kmin = nullptr;
    int nsplitK = 0, RK = 0;
    alignas(64) unsigned char tmapK[128] = {};
    bool tmapK_ok = false;
};

}  // namespace hobo

struct hobo_instance {
    int N = 0, order = 0, W = 0;
    int KF = 1, KU = 1, KS = 4;
    bool dense = false, integer = false;
    int64_t terms[HOBO_MAX_ORDER + 1] = {0};
    double abs_sum = 0.0;
    int device = 0;
    int num_sms = 0;
    int* status = nullptr;   // device status word written by kernels that give up a wait
    hobo::DevLayouts d;
    hobo_instance* low = nullptr;   // order-4 tensor-core instances: the degree <= 3 part
    bool owns_status = true;
};

namespace hobo {

// ---- kernel launchers (hobo_kernels.cu / hobo_tc.cu) ---------------------
cudaError_t launch_init_states(uint32_t* X, int B, int N, int W, uint64_t seed, cudaStream_t st,
                               uint32_t state0 = 0);

// g_or_dE: [B][N] or null; flip_out: write (1-2x)g instead of g
cudaError_t launch_energy_terms(const hobo_instance* h, const uint32_t* X, int B, float* E,
                                float* g_or_dE, bool flip_out, cudaStream_t st);

cudaError_t launch_energy_fp64(const hobo_instance* h, const uint32_t* X, int B, double* E,
                               cudaStream_t st);
// acc: device, B zeroed 64-bit accumulators owned by the caller
cudaError_t launch_energy_fp64_into(const hobo_instance* h, const uint32_t* X, int B, double* E,
                                    unsigned long long* acc, cudaStream_t st);

struct SweepArgs {
    int B = 0, sweeps = 0, sweep0 = 0, resume = 0, S = 32;
    uint64_t seed = 0;
    uint32_t state0 = 0;           // global index of state 0 (Philox counter offset)
    const float* beta = nullptr;   // device [sweeps]
    uint32_t* X = nullptr;         // device [B][W] in: start states, out: final
    float* g = nullptr;            // device [B][N] in: fields of X (plain: in/out)
    float* E = nullptr;            // device [B] in: energies of X, out: final
    uint32_t* bestX = nullptr;     // device [B][W]
    float* bestE = nullptr;        // device [B]
    int64_t* accepts = nullptr;    // device [B] or null
    int64_t* coef_bytes = nullptr; // device [B] or null
    bool write_g = false;          // tuned: write the final fields back to g
    float* vcache = nullptr;       // late-phase dense sweep: vector cache, or null
    int vslots = 0;                // its entries per state
};

cudaError_t launch_sweep_tuned(const hobo_instance* h, const SweepArgs& a, cudaStream_t st);
cudaError_t launch_sweep_plain(const hobo_instance* h, const SweepArgs& a, cudaStream_t st);

// tcgen05 dense order-3 contraction; returns cudaErrorNotSupported when the
// instance has no dense layout.
cudaError_t launch_energy_tc(const hobo_instance* h, const uint32_t* X, int B, float* E,
                             float* g_or_dE, bool flip_out, cudaStream_t st);
bool tc_supported(const hobo_instance* h);
bool exact_tc_supported(const hobo_instance* h);
bool fix_tc_supported(const hobo_instance* h);
cudaError_t make_tc_tensor_map_fl(hobo_instance* h);
// exact fixed-point energies and fields on the tensor cores (limb planes of
// the upper-triangular slabs), rounded once to float32
cudaError_t launch_energy_exact_f32(const hobo_instance* h, const uint32_t* X, int B, float* E, cudaStream_t st);
cudaError_t launch_energy_tc_fix(const hobo_instance* h, const uint32_t* X, int B, float* E, float* g_or_dE,
                                 bool flip_out, cudaStream_t st);
cudaError_t launch_wait_timeout_selftest(const hobo_instance* h, uint64_t limit_ns, cudaStream_t st);
cudaError_t make_tc_tensor_map(hobo_instance* h);
cudaError_t make_tc_tensor_map_rs(hobo_instance* h);
cudaError_t make_tc4_tensor_map(hobo_instance* h);
bool tc4_supported(const hobo_instance* h);
bool tck_supported(const hobo_instance* h);
cudaError_t make_tck_tensor_map(hobo_instance* h);
cudaError_t launch_energy_tck(const hobo_instance* h, const uint32_t* X, int B, float* E, float* g_or_dE,
                              bool flip_out, cudaStream_t st);
cudaError_t launch_energy_tc4(const hobo_instance* h, const uint32_t* X, int B, float* E, float* g_or_dE,
                              bool flip_out, cudaStream_t st);
cudaError_t launch_energy_exact_tc(const hobo_instance* h, const uint32_t* X, int B, unsigned long long* acc,
                                   cudaStream_t st);

// Forward pass of the proposal network on the tensor cores (hidden width
// 64..256, a multiple of 64): logits of the rows of F [n][3], or, with F
// null, of the score-table rows (sweep s, bit value x, point k) of beta [S]
// with G points over [-vmax, vmax].  Returns cudaErrorNotSupported for other
// widths.
bool mlp_tc_supported(int H);
cudaError_t launch_mlp_forward_tc(const float* w, int H, int64_t n, const float* F, const float* beta, int G,
                                  float vmax, float* out, int* status, cudaStream_t st);

void set_error(const std::string& msg);

// Runs an entry point's body so that no C++ exception crosses the C ABI: a
// failed host allocation returns HOBO_ERR_OOM, any other exception (e.g. a
// container length error from absurd sizes) HOBO_ERR_ARG, with a message.
template <class F>
int guarded(const char* what, F&& body)
{
    try {
        return body();
    } catch (const std::bad_alloc&) {
        set_error(std::string(what) + ": host allocation failed");
        return HOBO_ERR_OOM;
    } catch (const std::exception& e) {
        set_error(std::string(what) + ": " + e.what());
        return HOBO_ERR_ARG;
    } catch (...) {
        set_error(std::string(what) + ": unexpected error");
        return HOBO_ERR_ARG;
    }
}

// Energy/field contraction with the automatic or explicit path (0 auto,
// 1 term list, 2 tensor core exact, 3 tensor core with float32
// accumulation); returns a HOBO_* status.
int energy_dispatch(const hobo_instance* h, const uint32_t* X, int B, float* E, float* g, bool flip,
                    int path, cudaStream_t st);

}  // namespace hobo
