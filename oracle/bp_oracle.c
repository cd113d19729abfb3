/*
 * FP64 CPU oracle for frontier-based loopy belief propagation.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it. It shares no code, header, table or helper with the CUDA
 * library; the two meet only in the seeded input arrays.
 *
 * What it computes, step by step and in the paper's order:
 *   Eq. 1   pairwise MRF with psi_i = exp(theta_i), psi_ij = exp(theta_ij)
 *   Eq. 2   message update m_{i->j}(x_j) ~ sum_{x_i} psi_ij psi_i prod_{k in N(i)\j} m_{k->i}(x_i),
 *           computed in the probability domain, normalised to sum 1 (Section II-A:
 *           uniform initialisation, normalised between updates)
 *   Eq. 3   beliefs b_i(x_i) ~ psi_i(x_i) prod_{k in N(i)} m_{k->i}(x_i)
 *   Eq. 4   residual r(m_e) = ||f_BP(m)_e - m_e||, read as the max-norm over states
 *   Alg. 1  while not converged: frontier <- GenerateFrontier; Update(frontier); test
 *   Frontier generators:
 *     LBP   every message (Section II-B, Section III-A)
 *     RBP   top-k messages by residual, k = p * 2|E| (Section III-A, Section III-D)
 *     RS    top-k vertices by vertex residual (max incoming residual), then a splash
 *           (BFS of depth h) swept leaves -> root -> leaves (Section II-B, III-A, III-D)
 *     RnBP  residual >= eps filter, then a random fraction p of the rest, with p
 *           switched between LowP and HighP by EdgeRatio (Section IV-A, IV-D)
 *     RBP / RS with dynamic p: the same EdgeRatio switch sets their frontier
 *           fraction each round (Section IV-A, last sentence: tried there)
 *
 * Variable state counts (the protein-folding graphs of Section IV-E have 2 to
 * 81 states per vertex): a state whose unary log-potential is -inf is absent;
 * a message into a vertex is a distribution over its present states (uniform
 * at the start, no mass on absent states), which is Eq. 2 on the vertex's own
 * state space.
 *
 * Readings where the paper is silent (each one a named choice, shared with the
 * CUDA side only through its written description):
 *   residual norm = max over states of |candidate - current| of the normalised,
 *   probability-domain message; converged iff the max residual over all messages
 *   is strictly below eps; one round = evaluate all candidates and residuals,
 *   test, select, commit simultaneously (Jacobi); rounds = committing rounds;
 *   RBP/RS ties broken by smaller id; RBP k = clamp(ceil(p*M), 1, M); RS roots
 *   = clamp(ceil(p*M), 1, n) (or ceil(p*n) in the alternative mode); RnBP draws
 *   one 16-bit uniform per message -- half e mod 2 (0: low, 1: high) of word
 *   (e mod 8) / 2 of the Philox4x32-10 block with key seed and counter
 *   (floor(e / 8), round, graph, 0) -- and selects iff it is below
 *   floor(p * 2^16); EdgeRatio uses this round's and last round's unconverged
 *   counts, round 1 uses HighP.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LBP 0
#define ORC_RBP 1
#define ORC_RS 2
#define ORC_RNBP 3

#define ORC_PAIR_ISING 0
#define ORC_PAIR_TABLE 1
#define ORC_PAIR_SHARED 2

typedef struct {
    int32_t n, k;
    int64_t m;
    const int64_t *row_ptr;
    const int32_t *col;
    const int32_t *rev;
    const float *unary_log;  /* [n*k] */
    int32_t pair_kind;
    const float *pair_log;   /* Ising beta [m] | table [m*k*k] | shared [k*k] */
} orc_problem;

typedef struct {
    int32_t schedule;
    double parallelism;      /* p for RBP/RS, LowP for RnBP */
    double eps;
    int32_t max_rounds;
    uint64_t seed;
    uint32_t graph_id;
    double high_p;
    double ratio_threshold;
    int32_t splash_depth;
    int32_t rs_roots_mode;   /* 0: ceil(p*M) roots, 1: ceil(p*n) roots */
    const uint32_t *trace_in;  /* optional: frontier bitmask per round to follow */
    int32_t trace_rounds;
    uint32_t *trace_out;     /* optional: frontier bitmask per round, as selected */
    int32_t trace_cap;
    int32_t storage;         /* 0: exact FP64; 1: BF16 (Ising: the log-odds in the exponent
                                code below; other layouts: each log m(x) rounded);
                                2: 16-bit fixed-point log-odds (Ising only);
                                3: BF16 rounding of the plain Ising log-odds */
    double storage_scale;    /* storage 1 (Ising): log-odds per unit of log2 of the stored
                                word; storage 2: log-odds step of one integer unit */
    int32_t dynamic_p;       /* RBP / RS: 1 = frontier fraction by the EdgeRatio switch */
} orc_params;

typedef struct {
    int32_t converged, rounds;
    int64_t committed_updates, candidate_evals;
    double final_max_residual;
    int64_t final_unconverged;
} orc_stats;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): 10 rounds of the 4x32 S-box with multipliers 0xD2511F53 and
 * 0xCD9E8D57 and Weyl key increments 0x9E3779B9, 0xBB67AE85. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* RnBP random filter draw for message e in round t of graph g: one Philox
 * block per eight consecutive messages, counter (floor(e / 8), t, g, 0);
 * message e takes the 16-bit half e mod 2 (0: low, 1: high) of word
 * (e mod 8) / 2, a uniform integer in [0, 2^16). */
static uint32_t rnbp_draw(uint64_t seed, uint32_t e, uint32_t t, uint32_t g)
{
    uint32_t ctr[4] = {e / 8u, t, g, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    uint32_t word = out[(e % 8u) / 2u];
    return (e % 2u == 0u) ? (word & 0xffffu) : (word >> 16);
}

/* ------------------------------------------------------------------------- */
/* Model in the probability domain. Pairwise tables are indexed [e][x_src][x_dst]. */
typedef struct {
    const orc_problem *pb;
    int32_t *src;       /* [m] source vertex of each directed edge */
    double *psi_u;      /* [n*k] */
    uint8_t *present;   /* [n*k] 0 where the unary log-potential is -inf: an absent state */
    int32_t *k_present; /* [n] present states of each vertex */
    double *psi_p;      /* [m*k*k] (or [k*k] with stride 0 for the shared table) */
    int64_t pair_stride;
} orc_model;

static int model_init(orc_model *md, const orc_problem *pb)
{
    int32_t n = pb->n, k = pb->k;
    int64_t m = pb->m;
    memset(md, 0, sizeof(*md));
    md->pb = pb;
    md->psi_p = NULL;
    md->present = NULL;
    md->k_present = NULL;
    md->psi_u = NULL;
    md->src = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    md->psi_u = (double *)malloc(sizeof(double) * (size_t)n * (size_t)k + 8);
    md->present = (uint8_t *)malloc((size_t)n * (size_t)k + 8);
    md->k_present = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!md->src || !md->psi_u || !md->present || !md->k_present)
        return -1;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = pb->row_ptr[i]; e < pb->row_ptr[i + 1]; ++e)
            md->src[e] = i;
    for (int64_t q = 0; q < (int64_t)n * k; ++q) {
        md->psi_u[q] = exp((double)pb->unary_log[q]);
        md->present[q] = !(isinf(pb->unary_log[q]) && pb->unary_log[q] < 0.0f);
    }
    for (int32_t i = 0; i < n; ++i) {
        md->k_present[i] = 0;
        for (int32_t a = 0; a < k; ++a)
            md->k_present[i] += md->present[(int64_t)i * k + a];
    }
    if (pb->pair_kind == ORC_PAIR_SHARED) {
        md->pair_stride = 0;
        md->psi_p = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k);
        if (!md->psi_p)
            return -1;
        for (int64_t q = 0; q < (int64_t)k * k; ++q)
            md->psi_p[q] = exp((double)pb->pair_log[q]);
    } else {
        md->pair_stride = (int64_t)k * k;
        md->psi_p = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * (size_t)k * (size_t)k);
        if (!md->psi_p)
            return -1;
        for (int64_t e = 0; e < m; ++e) {
            for (int32_t a = 0; a < k; ++a) {
                for (int32_t b = 0; b < k; ++b) {
                    double theta;
                    if (pb->pair_kind == ORC_PAIR_ISING) {
                        double sa = (a == 0) ? -1.0 : 1.0, sb = (b == 0) ? -1.0 : 1.0;
                        theta = (double)pb->pair_log[e] * sa * sb;
                    } else {
                        theta = (double)pb->pair_log[e * k * k + (int64_t)a * k + b];
                    }
                    md->psi_p[e * k * k + (int64_t)a * k + b] = exp(theta);
                }
            }
        }
    }
    return 0;
}

static void model_free(orc_model *md)
{
    free(md->src);
    free(md->psi_u);
    free(md->present);
    free(md->k_present);
    free(md->psi_p);
}

/* Eq. 2 for one directed edge e = (i -> j), normalised; writes k values to c. */
static void message_update(const orc_model *md, const double *msg, int64_t e, double *c)
{
    const orc_problem *pb = md->pb;
    int32_t k = pb->k;
    int32_t i = md->src[e];
    const double *psi = md->psi_p + e * md->pair_stride;
    for (int32_t b = 0; b < k; ++b)
        c[b] = 0.0;
    for (int32_t a = 0; a < k; ++a) {
        double w = md->psi_u[(int64_t)i * k + a];
        for (int64_t f = pb->row_ptr[i]; f < pb->row_ptr[i + 1]; ++f) {
            if (f == e)
                continue;                     /* k ranges over N(i) \ j */
            w *= msg[(int64_t)pb->rev[f] * k + a];   /* m_{col[f] -> i}(x_i = a) */
        }
        for (int32_t b = 0; b < k; ++b)
            c[b] += psi[(int64_t)a * k + b] * w;
    }
    /* an absent state of j (unary log-potential -inf) carries no mass */
    int32_t j = pb->col[e];
    for (int32_t b = 0; b < k; ++b)
        if (!md->present[(int64_t)j * k + b])
            c[b] = 0.0;
    double z = 0.0;
    for (int32_t b = 0; b < k; ++b)
        z += c[b];
    for (int32_t b = 0; b < k; ++b)
        c[b] /= z;
}

/* Storage emulation. Messages may be kept in a 16-bit format; every value that
 * is committed then goes through the same rounding as the stored word, and
 * residuals compare rounded candidates with rounded current messages, so a
 * message whose stored value does not change has residual 0.
 *   BF16, Ising layout (k = 2, beta potentials): the stored word is the
 *   bfloat16 value nearest to w = 2^(|u| / b - 125), with the sign of the
 *   log-odds u = log m(1) - log m(0) and b = storage_scale. With b >= 2
 *   max|beta| / 250 every |u| <= 2 max|beta| maps into [2^-125, 2^125], so the
 *   word's 8 exponent bits and 7 mantissa bits form a logarithmic code of |u|
 *   whose step is at most b / 128 (a step of log2 w is at most 2^-7). The value is
 *   rounded to float, then to bfloat16, and read back as |u| = (log2 |w| +
 *   125) b.
 *   BF16 plain (storage 3, Ising layout): the log-odds itself rounded to float,
 *   then to bfloat16; its step is 2^-7 |u| (relative), which the exponent code
 *   above replaces by a uniform one.
 *   BF16, other layouts: log m(x) of each state rounded to bfloat16 (not
 *   renormalised after rounding).
 *   Q16: Ising log-odds rounded to the nearest multiple of storage_scale,
 *   clamped to +-32767 multiples.
 * Rounding to bfloat16 keeps 8 significant bits, to nearest, ties to even. */
static double round_bf16(double v)
{
    float f = (float)v;
    uint32_t b;
    memcpy(&b, &f, 4);
    b = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&f, &b, 4);
    return (double)f;
}

/* The value an Ising log-odds u is stored as: storage 0 keeps it, 1 codes it
 * in the exponent of a bfloat16 word, 2 rounds it to the nearest multiple of
 * the scale (ties to even) clamped to +-32767 multiples, 3 rounds it to
 * bfloat16. Exported so that tests can pin the rounding itself. */
double orc_stored_logodds(int32_t storage, double u, double scale)
{
    if (storage == 1) {
        double w = round_bf16(exp2(fabs(u) / scale - 125.0));
        double a = (log2(w) + 125.0) * scale;
        return u < 0.0 ? -a : a;
    }
    if (storage == 2) {
        double q = nearbyint(u / scale);
        if (q > 32767.0)
            q = 32767.0;
        if (q < -32767.0)
            q = -32767.0;
        return q * scale;
    }
    if (storage == 3)
        return round_bf16(u);
    return u;
}

static void store_round(const orc_problem *pb, const orc_params *pr, double *c)
{
    int32_t k = pb->k;
    if (pr->storage == 0)
        return;
    if (pb->pair_kind == ORC_PAIR_ISING) {
        double u = orc_stored_logodds(pr->storage, log(c[1]) - log(c[0]), pr->storage_scale);
        c[1] = 1.0 / (1.0 + exp(-u));
        c[0] = 1.0 / (1.0 + exp(u));
    } else {
        for (int32_t x = 0; x < k; ++x)
            c[x] = exp(round_bf16(log(c[x])));
    }
}

/* Eq. 4 with the max-norm. */
static double residual(const double *cand, const double *cur, int32_t k)
{
    double r = 0.0;
    for (int32_t b = 0; b < k; ++b) {
        double d = fabs(cand[b] - cur[b]);
        if (d > r)
            r = d;
    }
    return r;
}

/* Candidates (as they would be stored) and residuals of every message. */
static void evaluate_all(const orc_model *md, const orc_params *pr, const double *msg, double *cand,
                         double *r)
{
    const orc_problem *pb = md->pb;
    int32_t k = pb->k;
    for (int64_t e = 0; e < pb->m; ++e) {
        message_update(md, msg, e, cand + e * k);
        store_round(pb, pr, cand + e * k);
        r[e] = residual(cand + e * k, msg + e * k, k);
    }
}

/* Eq. 3. */
static void beliefs(const orc_model *md, const double *msg, double *out)
{
    const orc_problem *pb = md->pb;
    int32_t k = pb->k;
    for (int32_t i = 0; i < pb->n; ++i) {
        double z = 0.0;
        for (int32_t a = 0; a < k; ++a) {
            double w = md->psi_u[(int64_t)i * k + a];
            for (int64_t f = pb->row_ptr[i]; f < pb->row_ptr[i + 1]; ++f)
                w *= msg[(int64_t)pb->rev[f] * k + a];
            out[(int64_t)i * k + a] = w;
            z += w;
        }
        for (int32_t a = 0; a < k; ++a)
            out[(int64_t)i * k + a] /= z;
    }
}

/* ------------------------------------------------------------------------- */
/* Selection helpers. */

static const double *g_sort_key;   /* qsort has no context argument */

static int cmp_desc_then_id(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    double ka = g_sort_key[a], kb = g_sort_key[b];
    if (ka > kb)
        return -1;
    if (ka < kb)
        return 1;
    return (a < b) ? -1 : (a > b) ? 1 : 0;
}

/* Ids of the k largest keys, ties to the smaller id (stable descending sort). */
static void top_k(const double *key, int64_t count, int64_t k, int64_t *order_buf, uint8_t *chosen)
{
    if (count <= 0)
        return;
    for (int64_t q = 0; q < count; ++q)
        order_buf[q] = q;
    g_sort_key = key;
    qsort(order_buf, (size_t)count, sizeof(int64_t), cmp_desc_then_id);
    for (int64_t q = 0; q < count; ++q)
        chosen[q] = 0;
    for (int64_t q = 0; q < k && q < count; ++q)
        chosen[order_buf[q]] = 1;
}

static int64_t clamp_ceil(double p, int64_t base, int64_t lo, int64_t hi)
{
    double v = ceil(p * (double)base);
    int64_t k = (v > (double)hi) ? hi : (int64_t)v;
    if (k < lo)
        k = lo;
    if (k > hi)
        k = hi;
    return k;
}

/* Multi-source BFS over the undirected graph, level = distance to the nearest
 * root when <= depth, else -1. */
static void splash_levels(const orc_problem *pb, const uint8_t *root, int32_t depth,
                          int32_t *level, int32_t *queue)
{
    int64_t head = 0, tail = 0;
    for (int32_t v = 0; v < pb->n; ++v) {
        level[v] = -1;
        if (root[v]) {
            level[v] = 0;
            queue[tail++] = v;
        }
    }
    while (head < tail) {
        int32_t u = queue[head++];
        if (level[u] >= depth)
            continue;
        for (int64_t f = pb->row_ptr[u]; f < pb->row_ptr[u + 1]; ++f) {
            int32_t w = pb->col[f];
            if (level[w] < 0) {
                level[w] = level[u] + 1;
                queue[tail++] = w;
            }
        }
    }
}

static void trace_set(uint32_t *words, int64_t id)
{
    words[id >> 5] |= 1u << (id & 31);
}

static int trace_get(const uint32_t *words, int64_t id)
{
    return (int)((words[id >> 5] >> (id & 31)) & 1u);
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 with the four frontier generators.
 * Returns 0 on success, -1 on allocation failure, -2 on bad arguments. */
int orc_run(const orc_problem *pb, const orc_params *pr, double *beliefs_out,
            double *messages_out, orc_stats *st)
{
    if (!pb || !pr || pb->n < 0 || pb->k < 1 || pb->m < 0)
        return -2;
    if (pb->pair_kind == ORC_PAIR_ISING && pb->k != 2)
        return -2;
    int32_t n = pb->n, k = pb->k;
    int64_t m = pb->m;
    orc_model md;
    if (model_init(&md, pb) != 0) {
        model_free(&md);
        return -1;
    }
    size_t mk = (size_t)(m > 0 ? m : 1) * (size_t)k;
    double *msg = (double *)malloc(sizeof(double) * mk);
    double *cand = (double *)malloc(sizeof(double) * mk);
    double *r = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *vres = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)((m > n ? m : n) + 1));
    uint8_t *chosen = (uint8_t *)malloc((size_t)((m > n ? m : n) + 1));
    int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *tmp = (double *)malloc(sizeof(double) * (size_t)k);
    if (!msg || !cand || !r || !vres || !order || !chosen || !level || !queue || !tmp) {
        free(msg); free(cand); free(r); free(vres); free(order); free(chosen);
        free(level); free(queue); free(tmp);
        model_free(&md);
        return -1;
    }

    /* Section II-A: messages start uniform, over the present states of the
     * destination vertex. */
    for (int64_t e = 0; e < m; ++e) {
        int32_t j = pb->col[e];
        for (int32_t x = 0; x < k; ++x)
            msg[e * k + x] = md.present[(int64_t)j * k + x] ? 1.0 / (double)md.k_present[j] : 0.0;
    }
    for (int64_t e = 0; e < m; ++e)
        store_round(pb, pr, msg + e * k);

    int follow = (pr->trace_in != NULL);
    int64_t sel_count = (pr->schedule == ORC_RS) ? n : m;
    int64_t trace_words = (sel_count + 31) / 32;
    orc_stats s;
    memset(&s, 0, sizeof(s));
    int64_t n_prev = 0;
    int32_t t = 0;

    for (;;) {
        /* Evaluate: candidates and residuals of all messages (Eq. 2, Eq. 4). */
        evaluate_all(&md, pr, msg, cand, r);
        s.candidate_evals += m;
        double rmax = 0.0;
        int64_t n_t = 0;
        for (int64_t e = 0; e < m; ++e) {
            if (r[e] > rmax)
                rmax = r[e];
            if (r[e] >= pr->eps)
                ++n_t;
        }
        s.final_max_residual = rmax;
        s.final_unconverged = n_t;
        /* IsConverged (Alg. 1): strict max-residual test. */
        int converged_now = (rmax < pr->eps);
        if (follow) {
            if (t == pr->trace_rounds) {
                s.converged = converged_now;
                break;
            }
        } else {
            if (converged_now) {
                s.converged = 1;
                break;
            }
            if (t == pr->max_rounds)
                break;
        }
        t += 1;
        /* Parallelism of this round (Section IV-A): RnBP, and RBP / RS with
         * dynamic_p, switch between HighP (round 1, or EdgeRatio <= threshold)
         * and LowP (EdgeRatio = this round's unconverged count over the
         * previous round's > threshold); otherwise the fixed p. */
        double p_round = pr->parallelism;
        if (pr->schedule == ORC_RNBP || (pr->dynamic_p && pr->schedule != ORC_LBP)) {
            if (t == 1) {
                p_round = pr->high_p;
            } else {
                double ratio = (double)n_t / (double)n_prev;   /* EdgeRatio */
                p_round = (ratio > pr->ratio_threshold) ? pr->parallelism : pr->high_p;
            }
        }
        n_prev = n_t;
        const uint32_t *tin = follow ? pr->trace_in + (int64_t)(t - 1) * trace_words : NULL;
        uint32_t *tout = (pr->trace_out && t <= pr->trace_cap)
                             ? pr->trace_out + (int64_t)(t - 1) * trace_words : NULL;
        if (tout)
            memset(tout, 0, sizeof(uint32_t) * (size_t)trace_words);

        if (pr->schedule == ORC_RS) {
            /* Vertex residual = max residual over incoming messages. */
            for (int32_t v = 0; v < n; ++v)
                vres[v] = 0.0;
            for (int64_t e = 0; e < m; ++e)
                if (r[e] > vres[pb->col[e]])
                    vres[pb->col[e]] = r[e];
            if (follow) {
                for (int32_t v = 0; v < n; ++v)
                    chosen[v] = (uint8_t)trace_get(tin, v);
            } else {
                int64_t kv = pr->rs_roots_mode == 1 ? clamp_ceil(p_round, n, 1, n)
                                                    : clamp_ceil(p_round, m, 1, n);
                top_k(vres, n, kv, order, chosen);
            }
            if (tout)
                for (int32_t v = 0; v < n; ++v)
                    if (chosen[v])
                        trace_set(tout, v);
            splash_levels(pb, chosen, pr->splash_depth, level, queue);
            /* Sweep levels h, ..., 1, 0, 1, ..., h; each sub-step updates all
             * out-messages of that level's vertices from the messages current at
             * its start, then commits them together. */
            int32_t h = pr->splash_depth;
            for (int32_t step = 0; step <= 2 * h; ++step) {
                int32_t L = (step <= h) ? (h - step) : (step - h);
                int64_t touched = 0;
                for (int32_t v = 0; v < n; ++v) {
                    if (level[v] != L)
                        continue;
                    for (int64_t e = pb->row_ptr[v]; e < pb->row_ptr[v + 1]; ++e) {
                        message_update(&md, msg, e, cand + e * k);
                        store_round(pb, pr, cand + e * k);
                        ++touched;
                    }
                }
                for (int32_t v = 0; v < n; ++v) {
                    if (level[v] != L)
                        continue;
                    for (int64_t e = pb->row_ptr[v]; e < pb->row_ptr[v + 1]; ++e)
                        memcpy(msg + e * k, cand + e * k, sizeof(double) * (size_t)k);
                }
                s.candidate_evals += touched;
                s.committed_updates += touched;
            }
        } else {
            /* GenerateFrontier for LBP / RBP / RnBP. */
            if (follow) {
                for (int64_t e = 0; e < m; ++e)
                    chosen[e] = (uint8_t)trace_get(tin, e);
            } else if (pr->schedule == ORC_LBP) {
                for (int64_t e = 0; e < m; ++e)
                    chosen[e] = 1;
            } else if (pr->schedule == ORC_RBP) {
                top_k(r, m, clamp_ceil(p_round, m, 1, m), order, chosen);
            } else { /* RnBP */
                double p = p_round;
                int always = (p >= 1.0);
                uint64_t thr = (p <= 0.0) ? 0u : (uint64_t)(p * 65536.0);
                for (int64_t e = 0; e < m; ++e) {
                    chosen[e] = 0;
                    if (r[e] >= pr->eps) {                      /* eps filter */
                        uint32_t u = rnbp_draw(pr->seed, (uint32_t)e, (uint32_t)t, pr->graph_id);
                        if (always || (uint64_t)u < thr)        /* random filter */
                            chosen[e] = 1;
                    }
                }
            }
            /* Update(frontier): simultaneous commit of the selected candidates. */
            for (int64_t e = 0; e < m; ++e) {
                if (!chosen[e])
                    continue;
                memcpy(msg + e * k, cand + e * k, sizeof(double) * (size_t)k);
                s.committed_updates += 1;
                if (tout)
                    trace_set(tout, e);
            }
        }
    }
    s.rounds = t;

    if (beliefs_out)
        beliefs(&md, msg, beliefs_out);
    if (messages_out)
        memcpy(messages_out, msg, sizeof(double) * (size_t)m * (size_t)k);
    if (st)
        *st = s;
    (void)tmp;
    free(msg); free(cand); free(r); free(vres); free(order); free(chosen);
    free(level); free(queue); free(tmp);
    model_free(&md);
    return 0;
}

/* One evaluation from given messages: candidates [m*k] and residuals [m]. */
int orc_evaluate(const orc_problem *pb, const double *msg, double *cand, double *r)
{
    orc_model md;
    orc_params exact;
    memset(&exact, 0, sizeof(exact));
    if (model_init(&md, pb) != 0) {
        model_free(&md);
        return -1;
    }
    evaluate_all(&md, &exact, msg, cand, r);
    model_free(&md);
    return 0;
}

/* Eq. 3 from given messages. */
int orc_beliefs(const orc_problem *pb, const double *msg, double *out)
{
    orc_model md;
    if (model_init(&md, pb) != 0) {
        model_free(&md);
        return -1;
    }
    beliefs(&md, msg, out);
    model_free(&md);
    return 0;
}

/* Splash levels for given roots (exposed for the BFS pin). */
int orc_splash_levels(const orc_problem *pb, const uint8_t *root, int32_t depth, int32_t *level)
{
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(pb->n > 0 ? pb->n : 1));
    if (!queue)
        return -1;
    splash_levels(pb, root, depth, level, queue);
    free(queue);
    return 0;
}

/* Top-k selection (exposed for the selection pin). */
int orc_top_k(const double *key, int64_t count, int64_t k, uint8_t *chosen)
{
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(count + 1));
    if (!order)
        return -1;
    top_k(key, count, k, order, chosen);
    free(order);
    return 0;
}
