/*
 * CPU oracle for the HOBO energy contraction and the batched Metropolis
 * annealer (arXiv 2407.19987, "HOBOTAN").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain statement of what
 * the CUDA path computes.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (no contraction of a*b+c into FMA, no reassociation: every float
 * operation below is one IEEE round-to-nearest operation).
 *
 * Inputs are HOBO tensors in entry form: nnz index tuples of length
 * `order` (rows of idx) with one coefficient each, as in Sec. II.C; a
 * monomial of lower degree is stored with its smallest index repeated
 * (Sec. III.C), and binary variables satisfy x*x = x (Sec. II.B).
 *
 * Parity status of each routine (what pins it is in the tests):
 *   orc_energy*           pinned: brute force, x^T Q x, paper examples
 *   orc_flip_delta        pinned: definition (two evaluations)
 *   orc_fields            pinned: flip identity, Euler identity
 *   orc_philox4x32_10     pinned: published known-answer vectors
 *   orc_exp2              pinned: error bound against exp2 in fp64
 *   orc_anneal            pinned: equals orc_anneal_naive (re-evaluation)
 *                         on integer instances; ground states reached on
 *                         brute-forced instances.  The acceptance rule and
 *                         the random-number layout are readings (the paper
 *                         names simulated annealing only, Sec. II.D.1).
 *   orc_mlp_forward,      pinned: finite differences of the loss, networks
 *   orc_mlp_loss_grad     built to compute a known function, closed forms
 *                         of the loss at constant logits
 *   orc_anneal_learned    pinned: equals orc_anneal without a network and
 *                         with a constant network (ties by index); the set
 *                         of bits a learned sweep attempts equals the top
 *                         scores of the sweep's start state.  The proposal
 *                         itself has no counterpart in the paper.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ */
/* Energy by the definition of Sec. II.C / IV.C:                       */
/*   E(x) = sum over stored entries t of H_t * prod_d x[idx[t][d]]     */
/* ------------------------------------------------------------------ */

double orc_energy(const int32_t* idx, const double* coef, int64_t nnz, int order,
                  const uint8_t* x)
{
    double E = 0.0;
    for (int64_t t = 0; t < nnz; ++t) {
        int on = 1;
        for (int d = 0; d < order; ++d)
            if (!x[idx[t * order + d]]) { on = 0; break; }
        if (on) E += coef[t];
    }
    return E;
}

/* Batched form (Sec. IV.C): one energy per row of X (B rows of N bytes). */
void orc_energy_batch(const int32_t* idx, const double* coef, int64_t nnz, int order,
                      int N, const uint8_t* X, int64_t B, double* E)
{
    for (int64_t b = 0; b < B; ++b)
        E[b] = orc_energy(idx, coef, nnz, order, X + b * (int64_t)N);
}

/* Exact integer form for integer-coefficient instances. */
void orc_energy_batch_i64(const int32_t* idx, const int64_t* coef, int64_t nnz, int order,
                          int N, const uint8_t* X, int64_t B, int64_t* E)
{
    for (int64_t b = 0; b < B; ++b) {
        const uint8_t* x = X + b * (int64_t)N;
        int64_t acc = 0;
        for (int64_t t = 0; t < nnz; ++t) {
            int on = 1;
            for (int d = 0; d < order; ++d)
                if (!x[idx[t * order + d]]) { on = 0; break; }
            if (on) acc += coef[t];
        }
        E[b] = acc;
    }
}

/* Energy of every state 0..2^N-1 (bit i of the state number is x_i). */
void orc_bruteforce(const int32_t* idx, const double* coef, int64_t nnz, int order,
                    int N, double* Eall)
{
    uint8_t x[64];
    uint64_t total = (uint64_t)1 << N;
    for (uint64_t s = 0; s < total; ++s) {
        for (int i = 0; i < N; ++i) x[i] = (uint8_t)((s >> i) & 1u);
        Eall[s] = orc_energy(idx, coef, nnz, order, x);
    }
}

/* Flip deltas by definition: dE_i = E(x with bit i flipped) - E(x). */
void orc_flip_delta(const int32_t* idx, const double* coef, int64_t nnz, int order,
                    int N, const uint8_t* x, double* dE)
{
    uint8_t* y = (uint8_t*)malloc((size_t)N);
    memcpy(y, x, (size_t)N);
    double E0 = orc_energy(idx, coef, nnz, order, y);
    for (int i = 0; i < N; ++i) {
        y[i] ^= 1u;
        dE[i] = orc_energy(idx, coef, nnz, order, y) - E0;
        y[i] ^= 1u;
    }
    free(y);
}

/* Local fields of the multilinear objective: g_i = E(x|x_i=1) - E(x|x_i=0).
 * Computed term by term: an entry whose index set contains i contributes
 * its coefficient times the product of its other distinct variables. */
void orc_fields(const int32_t* idx, const double* coef, int64_t nnz, int order,
                int N, const uint8_t* x, double* g)
{
    for (int i = 0; i < N; ++i) g[i] = 0.0;
    for (int64_t t = 0; t < nnz; ++t) {
        const int32_t* r = idx + t * order;
        for (int d = 0; d < order; ++d) {
            int i = r[d];
            int seen = 0;
            for (int e = 0; e < d; ++e) if (r[e] == i) seen = 1;
            if (seen) continue;               /* each distinct member once */
            int on = 1;
            for (int e = 0; e < order; ++e)
                if (r[e] != i && !x[r[e]]) { on = 0; break; }
            if (on) g[i] += coef[t];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11): 10 rounds of the 4x32 Philox S-box     */
/* with the Weyl key schedule.                                          */
/* ------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t MA = 0xD2511F53u, MB = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t WA = 0x9E3779B9u, WB = 0xBB67AE85u;   /* Weyl increments */
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += WA; k1 += WB; }
        uint64_t pa = (uint64_t)MA * c0;
        uint64_t pb = (uint64_t)MB * c2;
        uint32_t hia = (uint32_t)(pa >> 32), loa = (uint32_t)pa;
        uint32_t hib = (uint32_t)(pb >> 32), lob = (uint32_t)pb;
        uint32_t n0 = hib ^ c1 ^ k0;
        uint32_t n1 = lob;
        uint32_t n2 = hia ^ c3 ^ k1;
        uint32_t n3 = loa;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------ */
/* exp2 of a non-positive float, specified as a fixed sequence of float */
/* operations so that two independent codes give identical bits:       */
/*   t < -125          -> 0                                             */
/*   n = floor(t + 0.5), f = t - n in [-0.5, 0.5]                       */
/*   p = degree-6 Taylor polynomial of 2^f = sum_k (ln 2)^k/k! f^k,     */
/*       coefficients rounded to the nearest float, Horner with         */
/*       separate multiply and add                                      */
/*   result = p * 2^n  (2^n built from its exponent field)              */
/* ------------------------------------------------------------------ */

static float f32_from_bits(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

float orc_exp2(float t)
{
    if (!(t >= -125.0f)) return 0.0f;
    float h = t + 0.5f;
    float n = floorf(h);
    float f = t - n;
    /* nearest float32 to (ln 2)^k / k!, k = 6..0 */
    float p = f32_from_bits(0x39218489u);
    p = p * f; p = p + f32_from_bits(0x3AAEC3FFu);
    p = p * f; p = p + f32_from_bits(0x3C1D955Bu);
    p = p * f; p = p + f32_from_bits(0x3D635847u);
    p = p * f; p = p + f32_from_bits(0x3E75FDF0u);
    p = p * f; p = p + f32_from_bits(0x3F317218u);
    p = p * f; p = p + 1.0f;
    int ni = (int)n;
    float s = f32_from_bits((uint32_t)(ni + 127) << 23);
    return p * s;
}

/* Metropolis acceptance for one attempted flip.  dE is the float flip
 * delta, beta the float inverse temperature, w a 32-bit Philox word.
 *   accept iff dE <= 0, or u < exp2(-(beta*dE) * log2(e))
 *   u = (w >> 8) * 2^-24 */
int orc_metropolis(float dE, float beta, uint32_t w)
{
    if (dE <= 0.0f) return 1;
    const float LOG2E = f32_from_bits(0x3FB8AA3Bu);     /* nearest float to 1/ln 2 */
    float a = beta * dE;
    float t = a * LOG2E;
    t = -t;
    float p = orc_exp2(t);
    float u = (float)(w >> 8) * (1.0f / 16777216.0f);
    return u < p;
}

/* Random-number layout (a reading; the paper specifies no generator):
 *   key     = (seed low 32 bits, seed high 32 bits)
 *   counter = (bit >> 2, sweep, state, stream), word (bit & 3)
 *   stream 1, sweep 0: initial bit = word >> 31
 *   stream 0, sweep s: Metropolis uniform of the attempt on that bit */
static uint32_t philox_word(uint64_t seed, uint32_t bit, uint32_t sweep, uint32_t state,
                            uint32_t stream)
{
    uint32_t ctr[4] = { bit >> 2, sweep, state, stream };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[bit & 3u];
}

void orc_init_states(uint64_t seed, int N, int64_t B, uint8_t* X)
{
    for (int64_t b = 0; b < B; ++b)
        for (int i = 0; i < N; ++i)
            X[b * N + i] = (uint8_t)(philox_word(seed, (uint32_t)i, 0u, (uint32_t)b, 1u) >> 31);
}

/* ------------------------------------------------------------------ */
/* Batched simulated annealing (Sec. II.D.1 names the method only; the  */
/* readings used here: single-bit Metropolis moves, bits visited in     */
/* order 0..N-1 once per sweep, inverse temperatures given per sweep,   */
/* the best state kept whenever the energy falls strictly below the     */
/* best so far).  States are independent.                               */
/*                                                                      */
/* orc_anneal keeps the fields g and the energy up to date after each   */
/* accepted flip: for every stored entry that contains the flipped bit  */
/* i, every other distinct member j gains delta * coef * (product of    */
/* the remaining members), delta = +1 for 0->1 and -1 for 1->0.         */
/* orc_anneal_naive instead re-evaluates E after each trial flip.       */
/* Both feed the float dE = (float)((1 - 2 x_i) g_i) to orc_metropolis. */
/*                                                                      */
/* Outputs per state: final bits and energy, best bits and energy,      */
/* accepted-flip count; optionally the bits of states < rec_B after     */
/* each sweep (rec: [sweeps][rec_B][N]).                                */
/* ------------------------------------------------------------------ */

typedef struct { int64_t* start; int64_t* list; } incidence_t;

static incidence_t build_incidence(const int32_t* idx, int64_t nnz, int order, int N)
{
    incidence_t inc;
    inc.start = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    for (int64_t t = 0; t < nnz; ++t)
        for (int d = 0; d < order; ++d) {
            int i = idx[t * order + d], seen = 0;
            for (int e = 0; e < d; ++e) if (idx[t * order + e] == i) seen = 1;
            if (!seen) inc.start[i + 1]++;
        }
    for (int i = 0; i < N; ++i) inc.start[i + 1] += inc.start[i];
    inc.list = (int64_t*)malloc((size_t)(inc.start[N] > 0 ? inc.start[N] : 1) * sizeof(int64_t));
    int64_t* fill = (int64_t*)malloc((size_t)N * sizeof(int64_t));
    for (int i = 0; i < N; ++i) fill[i] = inc.start[i];
    for (int64_t t = 0; t < nnz; ++t)
        for (int d = 0; d < order; ++d) {
            int i = idx[t * order + d], seen = 0;
            for (int e = 0; e < d; ++e) if (idx[t * order + e] == i) seen = 1;
            if (!seen) inc.list[fill[i]++] = t;
        }
    free(fill);
    return inc;
}

static void apply_flip(const int32_t* idx, const double* coef, int order,
                       const incidence_t* inc, uint8_t* x, double* g, int i)
{
    double delta = x[i] ? -1.0 : 1.0;     /* change of x_i */
    x[i] ^= 1u;
    for (int64_t p = inc->start[i]; p < inc->start[i + 1]; ++p) {
        int64_t t = inc->list[p];
        const int32_t* r = idx + t * order;
        for (int d = 0; d < order; ++d) {
            int j = r[d];
            if (j == i) continue;
            int seen = 0;
            for (int e = 0; e < d; ++e) if (r[e] == j) seen = 1;
            if (seen) continue;
            int on = 1;
            for (int e = 0; e < order; ++e)
                if (r[e] != i && r[e] != j && !x[r[e]]) { on = 0; break; }
            if (on) g[j] += delta * coef[t];
        }
    }
}

void orc_anneal(const int32_t* idx, const double* coef, int64_t nnz, int order, int N,
                uint64_t seed, int64_t state0, int64_t B, const float* betas, int sweeps,
                uint8_t* Xfinal, double* Efinal, uint8_t* Xbest, double* Ebest,
                int64_t* accepts, int64_t rec_B, uint8_t* rec)
{
    incidence_t inc = build_incidence(idx, nnz, order, N);
    uint8_t* x = (uint8_t*)malloc((size_t)N);
    double* g = (double*)malloc((size_t)N * sizeof(double));
    for (int64_t bb = 0; bb < B; ++bb) {
        uint32_t b = (uint32_t)(state0 + bb);
        for (int i = 0; i < N; ++i)
            x[i] = (uint8_t)(philox_word(seed, (uint32_t)i, 0u, b, 1u) >> 31);
        orc_fields(idx, coef, nnz, order, N, x, g);
        double E = orc_energy(idx, coef, nnz, order, x);
        double Eb = E;
        memcpy(Xbest + bb * N, x, (size_t)N);
        int64_t acc = 0;
        for (int s = 0; s < sweeps; ++s) {
            for (int i = 0; i < N; ++i) {
                float dE = (float)(x[i] ? -g[i] : g[i]);
                uint32_t w = philox_word(seed, (uint32_t)i, (uint32_t)s, b, 0u);
                if (orc_metropolis(dE, betas[s], w)) {
                    E += (x[i] ? -g[i] : g[i]);
                    apply_flip(idx, coef, order, &inc, x, g, i);
                    acc++;
                    if (E < Eb) { Eb = E; memcpy(Xbest + bb * N, x, (size_t)N); }
                }
            }
            if (rec && bb < rec_B)
                memcpy(rec + ((int64_t)s * rec_B + bb) * N, x, (size_t)N);
        }
        memcpy(Xfinal + bb * N, x, (size_t)N);
        Efinal[bb] = E;
        Ebest[bb] = Eb;
        accepts[bb] = acc;
    }
    free(g); free(x); free(inc.start); free(inc.list);
}

void orc_anneal_naive(const int32_t* idx, const double* coef, int64_t nnz, int order, int N,
                      uint64_t seed, int64_t state0, int64_t B, const float* betas, int sweeps,
                      uint8_t* Xfinal, double* Efinal, uint8_t* Xbest, double* Ebest,
                      int64_t* accepts)
{
    uint8_t* x = (uint8_t*)malloc((size_t)N);
    for (int64_t bb = 0; bb < B; ++bb) {
        uint32_t b = (uint32_t)(state0 + bb);
        for (int i = 0; i < N; ++i)
            x[i] = (uint8_t)(philox_word(seed, (uint32_t)i, 0u, b, 1u) >> 31);
        double E = orc_energy(idx, coef, nnz, order, x);
        double Eb = E;
        memcpy(Xbest + bb * N, x, (size_t)N);
        int64_t acc = 0;
        for (int s = 0; s < sweeps; ++s) {
            for (int i = 0; i < N; ++i) {
                x[i] ^= 1u;
                double E1 = orc_energy(idx, coef, nnz, order, x);
                x[i] ^= 1u;
                float dE = (float)(E1 - E);
                uint32_t w = philox_word(seed, (uint32_t)i, (uint32_t)s, b, 0u);
                if (orc_metropolis(dE, betas[s], w)) {
                    x[i] ^= 1u;
                    E = E1;
                    acc++;
                    if (E < Eb) { Eb = E; memcpy(Xbest + bb * N, x, (size_t)N); }
                }
            }
        }
        memcpy(Xfinal + bb * N, x, (size_t)N);
        Efinal[bb] = E;
        Ebest[bb] = Eb;
        accepts[bb] = acc;
    }
    free(x);
}

/* ------------------------------------------------------------------ */
/* Learned flip proposal: a small MLP scoring each bit from three        */
/* inputs (scaled local field, bit, temperature).  No counterpart in the */
/* paper; the architecture is 3 -> H -> H -> 1 with ReLU hidden layers, */
/* a logit output and binary cross-entropy against a 0/1 label:          */
/*   z1 = W1 f + b1, h1 = max(z1, 0)                                     */
/*   z2 = W2 h1 + b2, h2 = max(z2, 0)                                    */
/*   logit = w3 . h2 + b3                                                */
/*   loss = mean over rows of softplus(logit) - y * logit                */
/* Row-major weights: W1 [H][3], W2 [H][H] (row = output unit).          */
/* Gradients are of the mean loss, by the chain rule, in float64.        */
/* ------------------------------------------------------------------ */

static double relu(double v) { return v > 0.0 ? v : 0.0; }

static double softplus(double v)
{
    return v > 0.0 ? v + log1p(exp(-v)) : log1p(exp(v));
}

void orc_mlp_forward(int H, const double* W1, const double* b1, const double* W2, const double* b2,
                     const double* w3, double b3, const double* F, int64_t n, double* logit)
{
    double* h1 = (double*)malloc((size_t)H * sizeof(double));
    for (int64_t r = 0; r < n; ++r) {
        const double* f = F + r * 3;
        for (int u = 0; u < H; ++u)
            h1[u] = relu(W1[u * 3 + 0] * f[0] + W1[u * 3 + 1] * f[1] + W1[u * 3 + 2] * f[2] + b1[u]);
        double out = b3;
        for (int v = 0; v < H; ++v) {
            double z = b2[v];
            for (int u = 0; u < H; ++u) z += W2[(int64_t)v * H + u] * h1[u];
            out += w3[v] * relu(z);
        }
        logit[r] = out;
    }
    free(h1);
}

double orc_mlp_loss_grad(int H, const double* W1, const double* b1, const double* W2, const double* b2,
                         const double* w3, double b3, const double* F, const double* y, int64_t n,
                         double* gW1, double* gb1, double* gW2, double* gb2, double* gw3, double* gb3)
{
    double* z1 = (double*)malloc((size_t)H * sizeof(double));
    double* h1 = (double*)malloc((size_t)H * sizeof(double));
    double* z2 = (double*)malloc((size_t)H * sizeof(double));
    double* h2 = (double*)malloc((size_t)H * sizeof(double));
    double* d2 = (double*)malloc((size_t)H * sizeof(double));
    double* d1 = (double*)malloc((size_t)H * sizeof(double));
    memset(gW1, 0, sizeof(double) * (size_t)H * 3);
    memset(gb1, 0, sizeof(double) * (size_t)H);
    memset(gW2, 0, sizeof(double) * (size_t)H * H);
    memset(gb2, 0, sizeof(double) * (size_t)H);
    memset(gw3, 0, sizeof(double) * (size_t)H);
    *gb3 = 0.0;
    double loss = 0.0;
    for (int64_t r = 0; r < n; ++r) {
        const double* f = F + r * 3;
        for (int u = 0; u < H; ++u) {
            z1[u] = W1[u * 3 + 0] * f[0] + W1[u * 3 + 1] * f[1] + W1[u * 3 + 2] * f[2] + b1[u];
            h1[u] = relu(z1[u]);
        }
        double out = b3;
        for (int v = 0; v < H; ++v) {
            double z = b2[v];
            for (int u = 0; u < H; ++u) z += W2[(int64_t)v * H + u] * h1[u];
            z2[v] = z;
            h2[v] = relu(z);
            out += w3[v] * h2[v];
        }
        loss += softplus(out) - y[r] * out;
        /* d loss / d logit = sigmoid(logit) - y, divided by n for the mean */
        const double dl = (1.0 / (1.0 + exp(-out)) - y[r]) / (double)n;
        *gb3 += dl;
        for (int v = 0; v < H; ++v) {
            gw3[v] += dl * h2[v];
            d2[v] = z2[v] > 0.0 ? dl * w3[v] : 0.0;
            gb2[v] += d2[v];
        }
        for (int u = 0; u < H; ++u) d1[u] = 0.0;
        for (int v = 0; v < H; ++v) {
            if (d2[v] == 0.0) continue;
            for (int u = 0; u < H; ++u) {
                gW2[(int64_t)v * H + u] += d2[v] * h1[u];
                d1[u] += d2[v] * W2[(int64_t)v * H + u];
            }
        }
        for (int u = 0; u < H; ++u) {
            const double d = z1[u] > 0.0 ? d1[u] : 0.0;
            gW1[u * 3 + 0] += d * f[0];
            gW1[u * 3 + 1] += d * f[1];
            gW1[u * 3 + 2] += d * f[2];
            gb1[u] += d;
        }
    }
    free(z1); free(h1); free(z2); free(h2); free(d2); free(d1);
    return loss / (double)n;
}

/* ------------------------------------------------------------------ */
/* Annealing with the learned proposal (no counterpart in the paper).    */
/* Sweep s is plain (bits 0..N-1 in order, as orc_anneal) when there is  */
/* no network, when plain_every <= 1, or when s % plain_every ==         */
/* plain_every - 1.  Otherwise, at the start of the sweep every bit i is */
/* scored by the network on its features                                 */
/*   f0 = clamp(beta_s * g_i, -vmax, vmax) / 8                           */
/*   f1 = 2 x_i - 1,  f2 = -ln(beta_s) / 4                               */
/* (f0 in float32 from the float32 field, f1 exact, f2 in float64).      */
/* select 0: the bits are ordered by descending score with ties broken   */
/* by ascending index, and the first max(1, ceil(top_frac * N)) of them  */
/* are attempted in that order; select 1: the bits with score >=         */
/* threshold are attempted in index order.  Each attempt uses the same   */
/* Metropolis test and random word (bit i, sweep s) as a plain sweep.    */
/* Recording: for states b < rec_B and sweeps with s % rec_every == 0,   */
/* row (s / rec_every, b, i) gets the features of bit i at its decision  */
/* and its bit then (rec_x); rows of bits not attempted are left alone.  */
/* ------------------------------------------------------------------ */

typedef struct { double score; int i; } scored_t;

static int by_score_desc(const void* pa, const void* pb)
{
    const scored_t* a = (const scored_t*)pa;
    const scored_t* b = (const scored_t*)pb;
    if (a->score > b->score) return -1;
    if (a->score < b->score) return 1;
    return (a->i > b->i) - (a->i < b->i);
}

static float clampf_(float v, float lo, float hi) { return v < lo ? lo : (v > hi ? hi : v); }

void orc_anneal_learned(const int32_t* idx, const double* coef, int64_t nnz, int order, int N,
                        uint64_t seed, int64_t B, const float* betas, int sweeps,
                        int H, const double* W1, const double* b1, const double* W2, const double* b2,
                        const double* w3, double b3, int plain_every, int select, float top_frac,
                        double threshold, float vmax,
                        uint8_t* Xfinal, double* Efinal, uint8_t* Xbest, double* Ebest, int64_t* accepts,
                        int rec_every, int64_t rec_B, float* rec_F, uint8_t* rec_x)
{
    incidence_t inc = build_incidence(idx, nnz, order, N);
    uint8_t* x = (uint8_t*)malloc((size_t)N);
    double* g = (double*)malloc((size_t)N * sizeof(double));
    double* F = (double*)malloc((size_t)N * 3 * sizeof(double));
    double* sc = (double*)malloc((size_t)N * sizeof(double));
    scored_t* ord = (scored_t*)malloc((size_t)N * sizeof(scored_t));
    const int learned = W1 != NULL && plain_every > 1;
    for (int64_t b = 0; b < B; ++b) {
        for (int i = 0; i < N; ++i)
            x[i] = (uint8_t)(philox_word(seed, (uint32_t)i, 0u, (uint32_t)b, 1u) >> 31);
        orc_fields(idx, coef, nnz, order, N, x, g);
        double E = orc_energy(idx, coef, nnz, order, x);
        double Eb = E;
        memcpy(Xbest + b * N, x, (size_t)N);
        int64_t acc = 0;
        for (int s = 0; s < sweeps; ++s) {
            const float beta = betas[s];
            const double f2 = -log((double)beta) / 4.0;
            const int plain = !learned || (s % plain_every) == plain_every - 1;
            int nvisit = N;
            if (!plain) {
                for (int i = 0; i < N; ++i) {
                    float gi = (float)g[i];
                    float v = clampf_(beta * gi, -vmax, vmax);
                    F[i * 3 + 0] = (double)(v / 8.0f);
                    F[i * 3 + 1] = x[i] ? 1.0 : -1.0;
                    F[i * 3 + 2] = f2;
                }
                orc_mlp_forward(H, W1, b1, W2, b2, w3, b3, F, N, sc);
                if (select == 0) {
                    for (int i = 0; i < N; ++i) { ord[i].score = sc[i]; ord[i].i = i; }
                    qsort(ord, (size_t)N, sizeof(scored_t), by_score_desc);
                    float want = top_frac * (float)N;
                    nvisit = (int)ceilf(want);
                    if (nvisit > N) nvisit = N;
                    if (nvisit < 1) nvisit = 1;
                } else {
                    nvisit = 0;
                    for (int i = 0; i < N; ++i)
                        if (sc[i] >= threshold) ord[nvisit++].i = i;
                }
            }
            const int rec = rec_F && b < rec_B && (s % rec_every) == 0;
            const int64_t rbase = rec ? ((int64_t)(s / rec_every) * rec_B + b) * N : 0;
            for (int k = 0; k < nvisit; ++k) {
                const int i = plain ? k : ord[k].i;
                float gi = (float)g[i];
                float dE = x[i] ? -gi : gi;
                if (rec) {
                    float v = clampf_(beta * gi, -vmax, vmax);
                    rec_F[(rbase + i) * 3 + 0] = v / 8.0f;
                    rec_F[(rbase + i) * 3 + 1] = x[i] ? 1.0f : -1.0f;
                    rec_F[(rbase + i) * 3 + 2] = (float)f2;
                    rec_x[rbase + i] = x[i];
                }
                uint32_t w = philox_word(seed, (uint32_t)i, (uint32_t)s, (uint32_t)b, 0u);
                if (orc_metropolis(dE, beta, w)) {
                    E += (x[i] ? -g[i] : g[i]);
                    apply_flip(idx, coef, order, &inc, x, g, i);
                    acc++;
                    if (E < Eb) { Eb = E; memcpy(Xbest + b * N, x, (size_t)N); }
                }
            }
        }
        memcpy(Xfinal + b * N, x, (size_t)N);
        Efinal[b] = E;
        Ebest[b] = Eb;
        accepts[b] = acc;
    }
    free(ord); free(sc); free(F); free(g); free(x); free(inc.start); free(inc.list);
}
