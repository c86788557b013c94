/*
 * hobo.h -- C ABI of the GB300 HOBO contraction and annealing library.
 *
 * The library evaluates higher-order binary objectives stored as an order-k
 * HOBO tensor (arXiv 2407.19987, Sec. II.B-C) for a batch of binary states
 * (the tensor batch system of Sec. IV.C), and runs batched simulated
 * annealing over them (Sec. II.D.1).  All compute runs in the library's own
 * CUDA kernels for sm_103a.
 *
 * Conventions shared by every entry point:
 *  - Return value: HOBO_OK (0) or a negative HOBO_ERR_* code.  Nothing
 *    throws across the ABI.  hobo_last_error() returns a thread-local
 *    message describing the most recent failure on the calling thread.
 *  - Packed states: a state of N bits is W = ceil(N/32) uint32 words; bit i
 *    is bit (i % 32) of word (i / 32).  Bits at positions >= N in the last
 *    word are ignored on input and written as 0.
 *  - Device pointers are CUDA device (or managed) memory on the current
 *    device; host pointers are ordinary host memory.  The caller owns every
 *    buffer it passes; the library never frees or retains them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued asynchronously on it; host arrays passed
 *    to an entry point may be reused as soon as the call returns.
 *  - Energies exclude the constant term of the objective (the "offset" the
 *    paper's listings print, Sec. V): objective = energy + offset.
 */
#ifndef HOBO_H
#define HOBO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define HOBO_OK               0
#define HOBO_ERR_ARG         -1   /* null pointer, bad size, index out of range */
#define HOBO_ERR_ORDER       -2   /* order outside 1..HOBO_MAX_ORDER */
#define HOBO_ERR_NOT_EXACT   -3   /* HOBO_INTEGER requested but coefficients are
                                     not integers or sum |c| >= 2^24 */
#define HOBO_ERR_OOM         -4   /* device or host allocation failed */
#define HOBO_ERR_CUDA        -5   /* a CUDA runtime call failed */
#define HOBO_ERR_TIMEOUT     -6   /* a bounded device-side wait gave up */
#define HOBO_ERR_UNSUPPORTED -7   /* valid request this build does not cover */

#define HOBO_MAX_ORDER 8
#define HOBO_MAX_N     1024       /* variables per instance */

/* ---- creation flags -------------------------------------------------- */
#define HOBO_INTEGER      1u  /* require the bit-exact integer path: every folded
                                 coefficient an integer and sum |c| < 2^24, so
                                 every float32 partial sum is exact */
#define HOBO_FORCE_SPARSE 2u  /* use the term-list layouts even if dense */
#define HOBO_FORCE_DENSE  4u  /* build the dense slab layout (order <= 3) */
#define HOBO_SPLIT3       8u  /* tensor-core energy: always use the hi+mid+lo
                                 bf16 split (the default for non-integer
                                 coefficients; exact for float32 values) */
#define HOBO_SPLIT2      16u  /* tensor-core energy: hi+lo bf16 split for
                                 non-integer coefficients (relative error per
                                 coefficient <= 2^-16; faster, below the
                                 1e-5 bar on ill-conditioned fields).  Integer
                                 coefficients below 2^16 always use hi+lo,
                                 which is exact for them. */
#define HOBO_RESCORE_CUDA_CORES 32u  /* float64 re-score of dense instances on
                                 CUDA cores only (no limb planes for the
                                 exact tensor-core re-score; same results) */

typedef struct hobo_instance* hobo_h;

/*
 * hobo_create -- build an instance from a dense order-k tensor.
 *   T      host, float32, N^order entries, row-major (last index fastest).
 *          Any entry may be nonzero: an entry at index tuple t contributes
 *          T[t] * prod_{i in t} x_i.  Since x_i^2 = x_i for binary x, every
 *          entry is folded onto the distinct set of its indices (the
 *          replicate-smallest storage of Sec. III.C / IV.A is one case;
 *          entries below the diagonal are accepted too).
 *   order  1..HOBO_MAX_ORDER;  N 1..HOBO_MAX_N.
 *   flags  HOBO_* creation flags.
 * The tensor is copied; the caller keeps ownership of T.  Uses the current
 * CUDA device; synchronous.  N^order must fit in int64.
 * Errors: HOBO_ERR_ARG, HOBO_ERR_ORDER, HOBO_ERR_NOT_EXACT, HOBO_ERR_OOM,
 * HOBO_ERR_CUDA.  On error *out is set to NULL.
 */
int hobo_create(hobo_h* out, const float* T, int order, int N, unsigned flags);

/*
 * hobo_create_terms -- build an instance from tensor entries (Sec. II.C):
 *   idx   host int32 [nnz][order], each index in [0, N)
 *   coef  host float32 [nnz]
 * Entries with the same distinct index set are added (x^2 = x).  Same
 * ownership, flags and errors as hobo_create.
 */
int hobo_create_terms(hobo_h* out, const int32_t* idx, const float* coef, int64_t nnz,
                      int order, int N, unsigned flags);

/* Release an instance and all device memory it owns.  NULL is a no-op.
 * The caller must make sure no work using it is still in flight. */
void hobo_destroy(hobo_h h);

/* Static description of an instance (host-side, no GPU work). */
typedef struct {
    int N;                 /* variables */
    int order;             /* tensor order k */
    int words;             /* W = ceil(N/32) */
    int dense;             /* 1 if the dense slab layout is used */
    int integer;           /* 1 if all folded coefficients are integers and
                              sum |c| < 2^24 (bit-exact float32 path) */
    int64_t terms[HOBO_MAX_ORDER + 1];  /* folded monomials per degree */
    double abs_sum;        /* sum of |folded coefficient| */
    int tc_limbs;          /* dense order-3 instances: 8-bit limbs per
                              fixed-point coefficient in the exact
                              tensor-core contraction (0 = not built) */
} hobo_info_t;

int hobo_info(hobo_h h, hobo_info_t* info);

/*
 * hobo_energy -- batched contraction (Sec. IV.C): for each of B states,
 *   E[b]      = sum over folded monomials S of c_S * prod_{i in S} x_bi
 *   dE[b*N+i] = E(x_b with bit i flipped) - E(x_b) = (1 - 2 x_bi) g_bi,
 *               g_bi the local field dE/dx_i of the multilinear form.
 *   X   device uint32 [B][W] packed states
 *   E   device float32 [B]
 *   dE  device float32 [B][N], or NULL to skip the flip deltas
 * Dense order-3 instances (N <= 256) run the tcgen05 tensor-core
 * contraction: the tensor reshaped to (N^2 x N) rows (m, j) against the bit
 * matrix, upper triangle j < l of each slab only, on exact 8-bit limbs of
 * the fixed-point coefficients round(c * 2^S), integer sums, one rounding
 * to float32 (energies only: the re-score's m < j < l limbs).  Dense
 * order-4 instances with N <= 64 run the order-4 tensor-core contraction
 * (bf16 split, float32 accumulation); others the term-list kernel (exact
 * 64-bit fixed-point sums, one rounding).  Integer instances give exact
 * results on every path; the exact paths give identical floats.
 * B >= 0 (B = 0 is a no-op).  Errors: HOBO_ERR_ARG, HOBO_ERR_CUDA.
 */
int hobo_energy(hobo_h h, const uint32_t* X, int B, float* E, float* dE, void* stream);

/* hobo_energy with an explicit contraction path:
 *   path 0 = automatic, 1 = term-list kernel (CUDA cores, exact fixed point),
 *   path 2 = tcgen05 tensor-core kernel (dense order-3 instances: exact
 *            fixed-point limbs; dense order-4: bf16 split, float32 sums;
 *            HOBO_ERR_UNSUPPORTED otherwise),
 *   path 3 = tcgen05 kernel of dense order-3 instances on bf16 split
 *            planes of the full slabs with float32 accumulation (the
 *            Sec. IV.C contraction in plain tensor-core precision; float
 *            instances then carry float32 summation error; kept for
 *            comparison; HOBO_ERR_UNSUPPORTED otherwise). */
int hobo_energy_path(hobo_h h, const uint32_t* X, int B, float* E, float* dE, int path,
                     void* stream);

/*
 * hobo_energy_fp64 -- float64 energies of B packed states, for re-scoring
 * reported states.  The folded coefficients are held as exact 64-bit
 * fixed-point integers round(c * 2^S), S chosen per instance so that no
 * partial sum can overflow; each energy is the exact integer sum over the
 * active monomials, rounded once to float64.  Exact for integer instances;
 * otherwise the error is below that of a float64 summation.
 * X device uint32 [B][W]; E device double [B].
 */
int hobo_energy_fp64(hobo_h h, const uint32_t* X, int B, double* E, void* stream);

/*
 * hobo_energy_fp64_noalloc -- hobo_energy_fp64 that allocates nothing.
 * (The paper has no counterpart: this serves callers that cannot let the
 * library allocate device memory, e.g. applications whose GPU memory is
 * fully reserved by their own pool, or loops that must not risk an
 * allocation's synchronisation or pool growth.)
 *   Same arguments and results as hobo_energy_fp64, for B <= HOBO_NOALLOC_MAX_B
 *   states; larger B returns HOBO_ERR_ARG and does nothing.
 *   Scratch: a fixed 512 KiB array in device memory that every GPU loading
 *   the library holds until the process exits.  The first call on a device
 *   looks up that array's device address (make that first call before any
 *   stream capture).  Each call clears the part it uses, on `stream`.  All
 *   calls share the array: calls whose GPU work overlaps (other streams,
 *   no ordering) race and give wrong results, so order them.
 *   The instance must live on the current device (else HOBO_ERR_ARG).
 *   Errors: HOBO_ERR_ARG, HOBO_ERR_CUDA.
 */
#define HOBO_NOALLOC_MAX_B 65536
int hobo_energy_fp64_noalloc(hobo_h h, const uint32_t* X, int B, double* E, void* stream);

/* ---- annealing -------------------------------------------------------- */

#define HOBO_ANNEAL_TUNED  0  /* persistent kernel, states in shared memory */
#define HOBO_ANNEAL_PLAIN  1  /* one thread per state, fields in global memory */

typedef struct {
    int mode;              /* HOBO_ANNEAL_TUNED or HOBO_ANNEAL_PLAIN */
    int states_per_block;  /* tuned mode: 1..32 states per CTA, 0 = automatic */
    int sweep0;            /* index of the first sweep in the random stream
                              (resume: the number of sweeps already run) */
    int resume;            /* 1: start from X_io / bestX / bestE32_io instead of
                              the random initial states */
    uint32_t* X_io;        /* device [B][W] or NULL: start states when resume,
                              final states on return */
    float* bestE32_io;     /* device [B] or NULL: float32 best energy tracked
                              during the run (in when resume, out always) */
    float* E_io;           /* device [B] or NULL: final float32 energies on
                              return; with resume and g_io, the energies of
                              X_io to continue from */
    float* g_io;           /* device [B][N] or NULL: final float32 local fields
                              on return; with resume and E_io, the fields to
                              continue from (bit-exact continuation of a
                              float instance; without them fields and
                              energies are recomputed from X_io) */
    int64_t* accepts;      /* device [B] or NULL: accepted flips (added to) */
    int64_t* coef_bytes;   /* device [B] or NULL: bytes of coefficient data the
                              sweep read to update each state's fields after
                              its accepted flips (added to) */
    void* ev_sweep_begin;  /* cudaEvent_t or NULL: recorded on `stream` right
                              before the sweep kernel is enqueued */
    void* ev_sweep_end;    /* cudaEvent_t or NULL: recorded right after it */
    uint64_t state0;       /* global index of state 0 of this call: the random
                              streams of state b are those of state state0 + b,
                              so calls on disjoint index ranges (e.g. one per
                              GPU) reproduce one call on the whole range */
} hobo_anneal_opts;

/*
 * hobo_anneal -- batched Metropolis simulated annealing (Sec. II.D.1) of B
 * independent states.
 *   seed    64-bit key of the counter-based Philox4x32-10 stream.  The draw
 *           for (state b, sweep s, bit i) uses counter (i/4, s, b, 0),
 *           word i%4; initial bit i of state b uses counter (i/4, 0, b, 1),
 *           bit 31 of word i%4 (b offset by opts->state0, taken mod 2^32).
 *           Results do not depend on the launch shape.
 *   beta    host float32 [sweeps], inverse temperature of each sweep.
 *   Each sweep visits bits 0..N-1 in order; a flip with delta dE is
 *   accepted iff dE <= 0 or u < exp2(-(beta*dE)*log2 e), u = (w>>8)*2^-24,
 *   where exp2 is the library's fixed float sequence (range reduction to
 *   [-0.5,0.5], degree-6 Taylor polynomial; 0 below -125).  Fields are
 *   updated incrementally after each accepted flip; for a dense layout the
 *   vector added for a flip of bit i is S2[i] plus the float32 sum, in
 *   ascending order of the pairs (2q, 2q+1), of one slab row per pair with
 *   a listed bit (listed: the set bits other than i, or the clear ones with
 *   colsum[i] minus their sum when more than half are set), the
 *   pre-summed pair row where both are listed: the same floats in every
 *   mode and launch split.
 *   Temporaries are stream-ordered allocations on `stream` (schedule,
 *   states, fields; for dense layouts of up to 256 variables a cache of
 *   recent update vectors of at most 1 GiB, skipped when it cannot be had,
 *   from a memory pool of the library's that keeps up to 1 GiB per device
 *   between calls; the pool is made on the first dense anneal of a device
 *   and lives as long as the process: do not call cudaDeviceReset between
 *   anneals).
 *   bestX   device uint32 [B][W]: lowest-energy state seen by each state
 *           (strict improvement; in/out when opts->resume)
 *   bestE   device double [B]: energy of bestX re-scored in float64
 *   opts    NULL = tuned mode, fresh start
 * Integer instances follow the oracle's trajectories bit for bit.
 * Errors: HOBO_ERR_ARG, HOBO_ERR_OOM, HOBO_ERR_CUDA.
 */
int hobo_anneal(hobo_h h, uint64_t seed, int B, const float* beta, int sweeps,
                uint32_t* bestX, double* bestE, const hobo_anneal_opts* opts, void* stream);

/*
 * hobo_check -- wait for the work enqueued on `stream` and report whether
 * any kernel of this instance gave up a bounded device-side wait since the
 * last check (HOBO_ERR_TIMEOUT; the status is cleared).  Waits in the
 * library's kernels are time-limited, so a stall ends the kernel instead of
 * hanging the GPU.  Errors: HOBO_ERR_ARG, HOBO_ERR_CUDA, HOBO_ERR_TIMEOUT.
 */
int hobo_check(hobo_h h, void* stream);

/*
 * hobo_selftest_timeout -- diagnostic of the timeout path (no counterpart in
 * the paper): enqueues on `stream` a one-thread kernel that waits, through
 * the same bounded mbarrier wait as the contraction kernel, on a barrier
 * that nothing completes.  After limit_ns (1 .. 1e9 ns) the wait gives up
 * and records the timeout in h's status word, so the next hobo_check
 * returns HOBO_ERR_TIMEOUT (and clears it).  The GPU context stays usable.
 * Errors: HOBO_ERR_ARG (NULL h, limit out of range), HOBO_ERR_CUDA.
 */
int hobo_selftest_timeout(hobo_h h, uint64_t limit_ns, void* stream);

/*
 * hobo_selftest_philox -- diagnostic of the random stream (no counterpart in
 * the paper; the generator is Philox4x32-10 of Salmon et al., SC'11): for
 * each of n inputs, counter ctr[4i..4i+3] and key key[2i..2i+1] (device
 * arrays), writes the library's Philox4x32-10 block to ours[4i..4i+3] and
 * that of the CUDA toolkit's cuRAND device header (curand_Philox4x32_10) to
 * ref[4i..4i+3] (device arrays the caller owns).  The two must agree bit for
 * bit.  Errors: HOBO_ERR_ARG (n < 0, NULL array), HOBO_ERR_CUDA.
 */
int hobo_selftest_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* ours, uint32_t* ref,
                         void* stream);

/*
 * hobo_probe_l2_read -- measurement kernel with no counterpart in the paper:
 * enqueues on `stream` one launch that reads the device buffer `buf`
 * (`bytes` bytes, 16-byte aligned, a multiple of 16, at least 4096) `reps`
 * times in 16-byte loads cached in L2 only, from every SM (consecutive
 * threads read consecutive vectors; each thread steps through the buffer
 * with a stride of the grid's thread count, wrapping around).  With a
 * buffer that fits in L2 the caller's CUDA-event time of the launch gives
 * the GPU's L2-to-SM read bandwidth, bytes * reps / time: the denominator
 * of the sweep kernel's L2 roofline, since the sweep reads its coefficient
 * slabs out of L2.  Reads
 * only; writes nothing the caller sees.  Errors: HOBO_ERR_ARG (alignment,
 * size, reps outside 1..4096), HOBO_ERR_CUDA.
 */
int hobo_probe_l2_read(const void* buf, int64_t bytes, int reps, void* stream);

/* ---- batches of instances ---------------------------------------------- */

/*
 * A batch plan anneals many instances of uneven size together (the tensor
 * batch system of Sec. IV.C applied across instances).  It owns, per
 * instance t, B[t] states laid out in contiguous blocks: state block t
 * starts at state offset soff[t] = B[0] + ... + B[t-1] (energies) and at
 * word offset xoff[t] = sum_{u<t} B[u] * W_u (packed states, W_u =
 * ceil(N_u/32)); hobo_batch_layout returns both.  The instances must stay
 * alive while the plan exists.
 *
 * hobo_batch_anneal, mode HOBO_BATCH_GRAPH: the sweep of all instances runs
 * as one persistent kernel per layout kind (dense / sparse of order <= 3 /
 * order 4 / order 5..8) whose warps take (instance, state) items from a
 * queue sorted by decreasing cost; initial states, contraction, sweep and
 * re-score are captured once into a CUDA graph (rebuilt only when the
 * launch shape or the schedule buffer changes) and replayed on `stream`.
 * On the first call the launch shape (warps per CTA, CTAs per SM) is picked
 * by timing a few sweeps of each candidate (synchronous).  Modes
 * HOBO_BATCH_PER_INSTANCE_TUNED / _PLAIN run one launch sequence per
 * instance with the tuned / plain sweep instead.  In every mode state b of
 * instance t is annealed exactly as hobo_anneal(hs[t], seeds[t], ...) would
 * anneal state b.
 *   seeds  host [n];  beta host [sweeps]
 *   bestX  device, xoff[n-1] + B[n-1]*W_{n-1} words;  bestE device double
 *          [total states], float64 re-scored
 * Calls synchronise `stream` briefly to upload the instance descriptors.
 * Errors: HOBO_ERR_ARG, HOBO_ERR_OOM, HOBO_ERR_CUDA.
 */
typedef struct hobo_batch* hobo_batch_h;

#define HOBO_BATCH_GRAPH               0
#define HOBO_BATCH_PER_INSTANCE_TUNED  1
#define HOBO_BATCH_PER_INSTANCE_PLAIN  2

typedef struct {
    int mode;             /* HOBO_BATCH_* */
    int no_autotune;      /* 1: keep the current launch shape */
    int warps_per_cta;    /* > 0: force warps per CTA (1..8) */
    int ctas_per_sm;      /* > 0: force CTAs per SM */
    int64_t* accepts;     /* device [total] or NULL: accepted flips (added to) */
    uint32_t* X_out;      /* device, same layout as bestX, or NULL: final states */
    float* E_out;         /* device [total] or NULL: final float32 energies */
    void* ev_begin;       /* cudaEvent_t or NULL: recorded before the work */
    void* ev_end;         /* cudaEvent_t or NULL: recorded after the work */
} hobo_batch_opts;

int hobo_batch_create(hobo_batch_h* out, const hobo_h* hs, int n, const int* B);
void hobo_batch_destroy(hobo_batch_h bh);
int hobo_batch_layout(hobo_batch_h bh, int64_t* state_offset, int64_t* word_offset);
int hobo_batch_anneal(hobo_batch_h bh, const uint64_t* seeds, const float* beta, int sweeps,
                      uint32_t* bestX, double* bestE, const hobo_batch_opts* opts, void* stream);
/* Launch shape chosen for layout group `group` (0-based, in the order dense,
 * sparse order <= 3, order 4, order 5..8, skipping empty groups). */
int hobo_batch_launch_shape(hobo_batch_h bh, int group, int* warps_per_cta, int* ctas);

/* ---- learned flip proposal -------------------------------------------- */

/*
 * A small MLP scores each bit of a state from three features (no
 * counterpart in the paper; it is the learned part of the tuned annealer):
 *   f0 = clamp(beta * g_i, -vmax, vmax) / 8,  f1 = 2 x_i - 1,  f2 = -ln(beta) / 4
 * with g_i the bit's local field.  Network: 3 -> H -> H -> 1 (ReLU hidden
 * layers, logit output), bf16 weights, float32 sums; trained with binary
 * cross-entropy and Adam by the library's own kernels.  Flat parameter
 * layout (H = hidden): W1 [H][3] | b1 [H] | W2 [H][H] (row = output unit) |
 * b2 [H] | w3 [H] | b3.  All device pointers are on the current device.
 */
typedef struct hobo_mlp* hobo_mlp_h;

/* Create a network of hidden width H (multiple of 32, 32..1024) with He
 * initialisation from `seed`. */
int hobo_mlp_create(hobo_mlp_h* out, int hidden, uint64_t seed);
void hobo_mlp_destroy(hobo_mlp_h m);
int64_t hobo_mlp_num_params(hobo_mlp_h m);
/* Copy the parameters to host (rounded = 1: the bf16-rounded values the
 * passes use; 0: the float32 optimiser masters). */
int hobo_mlp_get(hobo_mlp_h m, float* host, int rounded);
/* Set the parameters from host float32 values (also resets Adam). */
int hobo_mlp_set(hobo_mlp_h m, const float* host);
/* Logits of n feature rows F (device [n][3]) into logit (device [n]).
 * Networks of hidden width 64..256 (a multiple of 64) run the H x H layer
 * on the tensor cores (tcgen05: hidden activations split into two bf16
 * planes hi + lo, relative residual <= 2^-16, against the bf16 weights,
 * float32 accumulation), with layer 1 and the head fused around it; other
 * widths run float32 CUDA-core passes.  The score tables of
 * hobo_anneal_learned use the same pass.  Errors: HOBO_ERR_ARG,
 * HOBO_ERR_CUDA; a device-side wait that gave up shows at hobo_mlp_check. */
int hobo_mlp_forward(hobo_mlp_h m, const float* F, int64_t n, float* logit, void* stream);
/* Score tables of the learned sweep: tables (device [S][2][G]) gets, for
 * sweep s (beta device [S]), bit value x and point k, the logit of the
 * features (v_k / 8, 2x - 1, -ln(beta_s) / 4), v_k = -vmax + 2 vmax k /
 * (G - 1) -- the table hobo_anneal_learned builds and interpolates.
 * Errors: HOBO_ERR_ARG (G outside 2..65536, vmax <= 0, NULL pointers),
 * HOBO_ERR_CUDA. */
int hobo_mlp_score_tables(hobo_mlp_h m, const float* beta, int S, int G, float vmax, float* tables, void* stream);
/* Choose the forward/table path: on = 1 tensor cores (the default where the
 * width allows it; HOBO_ERR_UNSUPPORTED otherwise), 0 CUDA-core passes.
 * Training passes always run on CUDA cores. */
int hobo_mlp_set_tensor_cores(hobo_mlp_h m, int on);
/* Wait for `stream` and report whether a network kernel gave up a bounded
 * device-side wait since the last check (HOBO_ERR_TIMEOUT; cleared). */
int hobo_mlp_check(hobo_mlp_h m, void* stream);
/* Mean binary cross-entropy of rows F against labels y (device [n], 0/1)
 * and its gradient w.r.t. the bf16-rounded parameters: grad device
 * [num_params] or NULL, loss device [1] or NULL. */
int hobo_mlp_loss_grad(hobo_mlp_h m, const float* F, const float* y, int64_t n, float* grad, float* loss,
                       void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on a mini-batch. */
int hobo_mlp_train_step(hobo_mlp_h m, const float* F, const float* y, int64_t n, float lr, float* loss,
                        void* stream);
/* Checkpoint: one JSON header line, then the bf16 parameters. */
int hobo_mlp_save(hobo_mlp_h m, const char* path);
int hobo_mlp_load(hobo_mlp_h* out, const char* path);

#define HOBO_SELECT_ORDER      0
#define HOBO_SELECT_THRESHOLD  1

typedef struct {
    int plain_every;     /* every plain_every-th sweep is plain (default 4);
                            <= 1: all sweeps plain (network unused) */
    int select;          /* HOBO_SELECT_ORDER (0): learned sweeps attempt the
                            top ceil(top_frac*N) bits in descending score
                            (ties by index); HOBO_SELECT_THRESHOLD (1): they
                            attempt, in index order, the bits whose score
                            (logit) is >= threshold */
    float top_frac;      /* order mode: fraction of bits attempted (0 = 1.0) */
    float threshold;     /* threshold mode: logit threshold */
    int table_size;      /* grid points of the per-sweep score table (0 = 256) */
    float vmax;          /* clamp of beta*g in the features (0 = 32) */
    int rec_every;       /* record sweeps s with s % rec_every == 0 (0: none) */
    int rec_states;      /* ... for states b < rec_states */
    float* rec_F;        /* device [ceil(sweeps/rec_every)][rec_states][N][3]: features */
    float* rec_y;        /* device [..][rec_states][N]: label 1 if the bit then
                            differs from the state's final best state, 0 if
                            not, -1 if the bit was not attempted */
    uint32_t* X_out;     /* device [B][W] or NULL: final states */
    float* E_out;        /* device [B] or NULL: final float32 energies */
    int64_t* accepts;    /* device [B] or NULL: accepted flips (added to) */
    void* ev_begin;      /* cudaEvent_t or NULL: recorded before the work */
    void* ev_end;        /* cudaEvent_t or NULL: recorded after the work */
} hobo_learned_opts;

/*
 * hobo_anneal_learned -- hobo_anneal with the learned proposal: in learned
 * sweeps each state scores its bits at the start of the sweep and attempts
 * either the top ceil(top_frac*N) of them in descending score (ties by
 * index) or those scoring >= threshold in index order (opts->select), with
 * the unchanged Metropolis test and random words; every plain_every-th
 * sweep is the plain sweep over all bits in order, which stays the
 * fallback.  Scores come from a
 * per-sweep table of the network over (clamped beta*g, bit), evaluated by
 * the library's forward kernel and read with linear interpolation.  m may
 * be NULL (all sweeps plain).  Requires N <= 256.  Same seed, beta, outputs
 * and errors as hobo_anneal; with all sweeps plain the results equal it.
 */
int hobo_anneal_learned(hobo_h h, hobo_mlp_h m, uint64_t seed, int B, const float* beta, int sweeps,
                        uint32_t* bestX, double* bestE, const hobo_learned_opts* opts, void* stream);

/* ---- tensor-train contraction ----------------------------------------- */

/*
 * A tensor in tensor-train form (Sec. VI): A[i1..id] = G_1[:, i1, :] ...
 * G_d[:, id, :] with cores G_c of shape [r_{c-1}][N][r_c], r_0 = r_d = 1 (the
 * successive-SVD decomposition of Sec. VI; the package's tt.py computes it).
 * hobo_tt_energy contracts the train with each state in every slot,
 * E(x) = sum over index tuples of A[i1..id] x_i1...x_id = M_1 ... M_d,
 * M_c = sum_i x_i G_c[:, i, :] (for a HOBO tensor: the energy of Sec. II.C),
 * at d*N*r^2 work per state instead of N^d.  Float32 sums.
 *   order 1..8, N 1..1024, ranks[0..order] host (interior ranks 1..256),
 *   cores host float32, the cores concatenated, core c row-major
 *   [r_{c-1}][N][r_c]; copied (caller keeps ownership).
 *   X device uint32 [B][ceil(N/32)] packed states; E device float [B].
 * Errors: HOBO_ERR_ARG, HOBO_ERR_ORDER, HOBO_ERR_OOM, HOBO_ERR_CUDA.
 */
typedef struct hobo_tt* hobo_tt_h;
int hobo_tt_create(hobo_tt_h* out, int order, int N, const int* ranks, const float* cores);
void hobo_tt_destroy(hobo_tt_h t);
int hobo_tt_energy(hobo_tt_h t, const uint32_t* X, int B, float* E, void* stream);

/* ---- result table ------------------------------------------------------ */

/*
 * hobo_aggregate -- the result table of a sampling run (Sec. V: states
 * listed by energy with their occurrence counts): the distinct states among
 * B packed states, sorted by energy ascending, ties by the lowest index at
 * which the state occurs.
 *   W      words per state (1..32), X device uint32 [B][W], E device double
 *          [B] (equal states must carry equal energies, as hobo_anneal's
 *          re-scored bestE do)
 *   U      device uint32 [B][W]: row r = r-th distinct state (first K rows)
 *   UE     device double [B]: its energy;  count device int64 [B]: how many
 *          of the B states equal it;  first device int32 [B]: its lowest index
 *   K      device int32 [1]: number of distinct states
 * Asynchronous on `stream`; scratch is stream-ordered.  The energies order
 * the table exactly as given (no tolerance): states whose energies differ in
 * the last bit are different rows.
 * Errors: HOBO_ERR_ARG, HOBO_ERR_CUDA.
 */
int hobo_aggregate(int W, const uint32_t* X, const double* E, int B, uint32_t* U, double* UE, int64_t* count,
                   int32_t* first, int32_t* K, void* stream);

/* Human-readable message of the last error on this thread ("" if none). */
const char* hobo_last_error(void);

/* Library version string. */
const char* hobo_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HOBO_H */
