/*
 * qcmet_oracle.c -- FP64 CPU oracle for layered sum-product syndrome decoding
 * of quasi-cyclic multi-edge-type LDPC codes (arXiv 2004.09084, Methods,
 * steps 1-4).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and is
 * loaded by the tests, by __graft_entry__.smoke() and by bench.py's CPU
 * baseline leg, nowhere else.  It shares no code, header, table or constant
 * generator with the CUDA decoder.  It is deliberately plain and slow: one
 * check node at a time, in the order the paper states, in double precision.
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *  - Circulant convention (Results, Eq. (m) and the sentence after it): a base
 *    entry a is the identity shifted right by a, so check l*Z+i touches
 *    variable c*Z + (i+a) mod Z.
 *  - Order inside one layer (Results, description of the fused kernel, and
 *    Methods step 3): q = L_qn - L_rmn(old) is formed first, the check rule of
 *    step 2 runs on those q, then L_qn = q + L_rmn(new).
 *  - Clipping (Results, paragraph on the kernel's API calls; constants not
 *    given): the argument of every Phi is clipped to [PHI(30), 30].  Phi maps
 *    that interval onto itself, so every |L_rmn| lies in [PHI(30), 30].
 *  - sgn(x) = -1 for x < 0 and +1 otherwise (so sgn(+-0) = +1), matching the
 *    hard-decision tie rule of step 4 (L >= 0 -> bit 0).
 *  - Phi(x) = -ln tanh(x/2) is evaluated as log1p(2 / expm1(x)), the same
 *    function written so that it keeps full relative precision at both ends
 *    of the clipping interval.
 *  - Degree-1 variables are updated like every other variable (no shortcut).
 *
 * Parity pins: every function here is checked by tests against results that
 * the paper or the mathematics fixes (brute-force check marginals, exact APP
 * marginals on cycle-free codes, closed forms and invariants).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_CLIP_MAX 30.0

/* check-node rules */
#define ORACLE_RULE_PHI 0      /* Methods step 2: Phi-sum form (the paper's rule) */
#define ORACLE_RULE_TANH 1     /* 2 atanh(prod tanh(q/2)): the same rule, cross-check only */
#define ORACLE_RULE_MINSUM 2   /* offset/scaled min-sum with per-(type, layer, iteration) weights */

/* message storage formats (the C2V messages L_rmn are rounded on store) */
#define ORACLE_MSG_EXACT 0
#define ORACLE_MSG_FP16 1
#define ORACLE_MSG_BF16 2

/* ---------------------------------------------------------------------- */
/* Phi(x) = -ln(tanh(x/2)), Methods step 2.  Phi is its own inverse.       */

static double phi_unclipped(double x)
{
    return log1p(2.0 / expm1(x));
}

double oracle_clip_min(void)
{
    return phi_unclipped(ORACLE_CLIP_MAX);
}

double oracle_clip_max(void)
{
    return ORACLE_CLIP_MAX;
}

double oracle_phi(double x)
{
    const double lo = phi_unclipped(ORACLE_CLIP_MAX);
    if (x < lo) x = lo;
    if (x > ORACLE_CLIP_MAX) x = ORACLE_CLIP_MAX;
    return phi_unclipped(x);
}

static double sgn(double x)
{
    return x < 0.0 ? -1.0 : 1.0;
}

/* Round x to the nearest value of a binary format with p significand bits and
 * minimum normal exponent emin (ties to even; subnormals keep the quantum of
 * the minimum exponent).  IEEE 754 round-to-nearest written out. */
static double round_to_format(double x, int p, int emin)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(x, &e);          /* x = f * 2^e with 0.5 <= |f| < 1 */
    int E = e - 1;         /* unit exponent: 2^E <= |x| < 2^(E+1) */
    if (E < emin) E = emin;
    double quantum = ldexp(1.0, E - (p - 1));
    return nearbyint(x / quantum) * quantum;
}

static double store_msg(double r, int fmt)
{
    switch (fmt) {
    case ORACLE_MSG_FP16: return round_to_format(r, 11, -14);
    case ORACLE_MSG_BF16: return round_to_format(r, 8, -126);
    default: return r;
    }
}

double oracle_round_msg(double r, int fmt)
{
    return store_msg(r, fmt);
}

/* ---------------------------------------------------------------------- */
/* Step 2 for one check node of degree d.                                  */
/*   q[j]  : variable-to-check messages L_qnm of the check's d edges       */
/*   s     : syndrome bit s_m                                              */
/*   r[j]  : out, check-to-variable messages L_rmn                         */
/* The exclusive sums over N(m)\n are formed directly, edge by edge.       */

static void check_phi(int d, const double *q, int s, double *r)
{
    for (int j = 0; j < d; ++j) {
        double sign = 1.0;
        double sum = 0.0;
        for (int k = 0; k < d; ++k) {
            if (k == j) continue;
            sign *= sgn(q[k]);
            sum += oracle_phi(fabs(q[k]));
        }
        double mag = oracle_phi(sum);      /* Phi^{-1} = Phi */
        r[j] = (s ? -1.0 : 1.0) * sign * mag;
    }
}

static void check_tanh(int d, const double *q, int s, double *r)
{
    const double lo = oracle_clip_min();
    for (int j = 0; j < d; ++j) {
        double prod = 1.0;
        for (int k = 0; k < d; ++k) {
            if (k == j) continue;
            double a = fabs(q[k]);
            if (a < lo) a = lo;
            if (a > ORACLE_CLIP_MAX) a = ORACLE_CLIP_MAX;
            prod *= sgn(q[k]) * tanh(0.5 * a);
        }
        double mag = 2.0 * atanh(fabs(prod));
        if (mag < lo) mag = lo;
        if (mag > ORACLE_CLIP_MAX) mag = ORACLE_CLIP_MAX;
        r[j] = (s ? -1.0 : 1.0) * sgn(prod) * mag;
    }
}

/* Offset/scaled min-sum: |r| = min(max(w_scale * min_{k != j} |q_k| - w_offset, 0), 30),
 * sign as in step 2.  (Learned variant; not part of the paper's method.  The
 * upper clip is the one the sum-product rule uses: without it, unscaled
 * min-sum can grow posteriors geometrically past the FP32 range.) */
static void check_minsum(int d, const double *q, int s, const double *w_scale,
                         const double *w_offset, double *r)
{
    for (int j = 0; j < d; ++j) {
        double sign = 1.0;
        double mn = INFINITY;
        for (int k = 0; k < d; ++k) {
            if (k == j) continue;
            sign *= sgn(q[k]);
            double a = fabs(q[k]);
            if (a < mn) mn = a;
        }
        if (d == 1) mn = ORACLE_CLIP_MAX;
        double mag = w_scale[j] * mn - w_offset[j];
        if (mag < 0.0) mag = 0.0;
        if (mag > ORACLE_CLIP_MAX) mag = ORACLE_CLIP_MAX;
        r[j] = (s ? -1.0 : 1.0) * sign * mag;
    }
}

void oracle_check_update(int d, const double *q, int s, int rule, double *r)
{
    if (rule == ORACLE_RULE_TANH) check_tanh(d, q, s, r);
    else check_phi(d, q, s, r);
}

/* ---------------------------------------------------------------------- */
/* The Tanner graph of the expanded code.                                  */

typedef struct {
    int mb, nb, Z;
    int n_circ;          /* number of circulants (non-zero base entries)    */
    int *row_first;      /* [mb+1] first circulant of each base row          */
    int *circ_col;       /* [n_circ] base column of each circulant           */
    int *circ_shift;     /* [n_circ] shift a of each circulant               */
    int *circ_type;      /* [n_circ] edge type (for the learned rule)       */
    int max_deg;
} graph_t;

static void graph_free(graph_t *g)
{
    free(g->row_first);
    free(g->circ_col);
    free(g->circ_shift);
    free(g->circ_type);
}

/* returns 0 on success, <0 on invalid input */
static int graph_build(int mb, int nb, int Z, const int8_t *base, const int32_t *shifts,
                       graph_t *g)
{
    memset(g, 0, sizeof(*g));
    if (mb < 1 || nb < 1 || Z < 1) return -1;
    g->mb = mb;
    g->nb = nb;
    g->Z = Z;
    int n_circ = 0;
    for (int i = 0; i < mb * nb; ++i) n_circ += base[i] != 0;
    g->n_circ = n_circ;
    g->row_first = (int *)malloc(sizeof(int) * (size_t)(mb + 1));
    g->circ_col = (int *)malloc(sizeof(int) * (size_t)(n_circ + 1));
    g->circ_shift = (int *)malloc(sizeof(int) * (size_t)(n_circ + 1));
    g->circ_type = (int *)malloc(sizeof(int) * (size_t)(n_circ + 1));
    if (!g->row_first || !g->circ_col || !g->circ_shift || !g->circ_type) {
        graph_free(g);
        return -2;
    }
    /* column degrees (number of circulants in each base column) */
    int *coldeg = (int *)calloc((size_t)nb, sizeof(int));
    if (!coldeg) {
        graph_free(g);
        return -2;
    }
    for (int l = 0; l < mb; ++l)
        for (int c = 0; c < nb; ++c) coldeg[c] += base[l * nb + c] != 0;
    int k = 0;
    g->max_deg = 0;
    for (int l = 0; l < mb; ++l) {
        g->row_first[l] = k;
        for (int c = 0; c < nb; ++c) {
            if (!base[l * nb + c]) continue;
            int a = shifts[l * nb + c];
            if (a < 0 || a >= Z) {
                free(coldeg);
                graph_free(g);
                return -3;
            }
            g->circ_col[k] = c;
            g->circ_shift[k] = a;
            g->circ_type[k] = coldeg[c] == 1 ? 1 : 0;   /* 1: edge to a degree-1 variable */
            ++k;
        }
        int d = k - g->row_first[l];
        if (d > g->max_deg) g->max_deg = d;
    }
    g->row_first[mb] = k;
    free(coldeg);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Step 4 and the syndrome test: hard decisions from L_qn, 1 iff H c = s.  */

static int hard_and_test(const graph_t *g, const double *Lq, const uint8_t *syn, uint8_t *hard)
{
    const int Z = g->Z;
    const int n = g->nb * Z;
    for (int i = 0; i < n; ++i) hard[i] = Lq[i] >= 0.0 ? 0 : 1;   /* c_n = 0 iff L_qn >= 0 */
    for (int l = 0; l < g->mb; ++l) {
        const int c0 = g->row_first[l];
        const int d = g->row_first[l + 1] - c0;
        for (int i = 0; i < Z; ++i) {
            int par = syn[l * Z + i] & 1;
            for (int j = 0; j < d; ++j) {
                const int k = c0 + j;
                par ^= hard[g->circ_col[k] * Z + (i + g->circ_shift[k]) % Z];
            }
            if (par) return 0;
        }
    }
    return 1;
}

/* ---------------------------------------------------------------------- */
/* One frame of layered BP, steps 1-4.                                     */

typedef struct {
    const graph_t *g;
    const int32_t *order;   /* base rows in processing order */
    int n_order;
    int T;
    int rule;
    int msg_fmt;
    const double *w_scale;  /* min-sum weights [T][mb][2] or NULL */
    const double *w_offset;
    int early_every;        /* > 0: test H c = s after every early_every-th iteration */
} decode_cfg_t;

static int decode_frame(const decode_cfg_t *cfg, const float *llr_ch, const uint8_t *syn,
                        uint8_t *hard, double *llr_post, uint8_t *ok, int32_t *iters_used)
{
    const graph_t *g = cfg->g;
    const int Z = g->Z;
    const int n = g->nb * Z;
    const size_t E = (size_t)g->n_circ * (size_t)Z;
    double *Lq = (double *)malloc(sizeof(double) * (size_t)n);   /* L_qn     */
    double *Lr = (double *)calloc(E ? E : 1, sizeof(double));     /* L_rmn    */
    int d_max = g->max_deg > 0 ? g->max_deg : 1;
    double *q = (double *)malloc(sizeof(double) * (size_t)d_max);  /* L_qnm    */
    double *r = (double *)malloc(sizeof(double) * (size_t)d_max);
    double *ws = (double *)malloc(sizeof(double) * (size_t)d_max);
    double *wo = (double *)malloc(sizeof(double) * (size_t)d_max);
    int *v = (int *)malloc(sizeof(int) * (size_t)d_max);
    if (!Lq || !Lr || !q || !r || !v || !ws || !wo) {
        free(Lq); free(Lr); free(q); free(r); free(v); free(ws); free(wo);
        return -2;
    }

    /* step 1: L_qn = 2 R_n / sigma^2, supplied as the channel LLR */
    for (int i = 0; i < n; ++i) Lq[i] = (double)llr_ch[i];

    int t_used = cfg->T;
    int stopped = 0;
    for (int t = 0; t < cfg->T && !stopped; ++t) {
        for (int oi = 0; oi < cfg->n_order; ++oi) {
            const int l = cfg->order[oi];
            const int c0 = g->row_first[l];
            const int d = g->row_first[l + 1] - c0;
            for (int i = 0; i < Z; ++i) {
                const int m = l * Z + i;
                /* step 3, first equation: L_qnm = L_qn - L_rmn(old) */
                for (int j = 0; j < d; ++j) {
                    const int k = c0 + j;
                    v[j] = g->circ_col[k] * Z + (i + g->circ_shift[k]) % Z;
                    q[j] = Lq[v[j]] - Lr[(size_t)k * Z + i];
                }
                /* step 2: check-to-variable messages with the syndrome sign */
                if (cfg->rule == ORACLE_RULE_MINSUM) {
                    for (int j = 0; j < d; ++j) {
                        const int typ = g->circ_type[c0 + j];
                        const size_t wi = ((size_t)t * g->mb + l) * 2 + typ;
                        ws[j] = cfg->w_scale[wi];
                        wo[j] = cfg->w_offset[wi];
                    }
                    check_minsum(d, q, syn[m], ws, wo, r);
                } else {
                    oracle_check_update(d, q, syn[m], cfg->rule, r);
                }
                /* step 3, second equation: L_qn = L_qnm + L_rmn(new) */
                for (int j = 0; j < d; ++j) {
                    const int k = c0 + j;
                    const double rs = store_msg(r[j], cfg->msg_fmt);
                    Lr[(size_t)k * Z + i] = rs;
                    Lq[v[j]] = q[j] + rs;
                }
            }
        }
        /* early termination (Discussion, Table tabearly): stop once H c = s */
        if (cfg->early_every > 0 && (t + 1) % cfg->early_every == 0 && t + 1 < cfg->T &&
            hard_and_test(g, Lq, syn, hard)) {
            t_used = t + 1;
            stopped = 1;
        }
    }

    /* step 4: hard decision, c_n = 0 iff L_qn >= 0, and the syndrome flag */
    *ok = (uint8_t)hard_and_test(g, Lq, syn, hard);
    if (llr_post)
        for (int i = 0; i < n; ++i) llr_post[i] = Lq[i];
    if (iters_used) *iters_used = t_used;
    free(Lq); free(Lr); free(q); free(r); free(v); free(ws); free(wo);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Threads over frames (frames are independent).                           */

typedef struct {
    const decode_cfg_t *cfg;
    int K, n, m;
    const float *llr_ch;
    const uint8_t *syn;
    uint8_t *hard;
    double *llr_post;
    uint8_t *ok;
    int32_t *iters_used;
    int tid, nthreads;
    int status;
} worker_t;

static void *worker_main(void *arg)
{
    worker_t *w = (worker_t *)arg;
    w->status = 0;
    for (int k = w->tid; k < w->K; k += w->nthreads) {
        int st = decode_frame(w->cfg, w->llr_ch + (size_t)k * w->n, w->syn + (size_t)k * w->m,
                              w->hard + (size_t)k * w->n,
                              w->llr_post ? w->llr_post + (size_t)k * w->n : NULL, w->ok + k,
                              w->iters_used ? w->iters_used + k : NULL);
        if (st) {
            w->status = st;
            break;
        }
    }
    return NULL;
}

/*
 * Decode K frames.
 *   base, shifts : [mb*nb] row-major base matrix (non-zero = circulant) and shifts
 *   order        : base rows in processing order (NULL = 0..mb-1); may list a
 *                  subset or repeat rows only if the caller wants that schedule
 *   llr_ch       : [K][n] channel LLRs, syn: [K][m] syndrome bits
 *   hard, ok     : outputs [K][n] and [K]; llr_post: [K][n] or NULL
 *   rule         : ORACLE_RULE_*; msg_fmt: ORACLE_MSG_*
 *   w_scale, w_offset : min-sum weights [T][mb][2] (type 0: edge to a variable
 *                  of degree > 1, type 1: edge to a degree-1 variable), or NULL
 *   early_every  : > 0 tests H c = s after every early_every-th iteration and
 *                  stops a frame that passes; 0 runs all T iterations
 *   iters_used   : [K] iterations each frame ran, or NULL
 * Returns 0, or <0 on invalid input / allocation failure.
 */
int oracle_decode(int mb, int nb, int Z, const int8_t *base, const int32_t *shifts,
                  const int32_t *order, int n_order, int K, int T, const float *llr_ch,
                  const uint8_t *syn, uint8_t *hard, double *llr_post, uint8_t *ok, int rule,
                  int msg_fmt, const double *w_scale, const double *w_offset, int nthreads,
                  int early_every, int32_t *iters_used)
{
    if (K < 0 || T < 0 || !base || !shifts || (K > 0 && (!llr_ch || !syn || !hard || !ok)))
        return -1;
    if (rule == ORACLE_RULE_MINSUM && (!w_scale || !w_offset)) return -1;
    graph_t g;
    int st = graph_build(mb, nb, Z, base, shifts, &g);
    if (st) return st;
    int32_t *ord = NULL;
    if (!order) {
        ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)mb);
        if (!ord) {
            graph_free(&g);
            return -2;
        }
        for (int l = 0; l < mb; ++l) ord[l] = l;
        order = ord;
        n_order = mb;
    } else {
        for (int i = 0; i < n_order; ++i)
            if (order[i] < 0 || order[i] >= mb) {
                graph_free(&g);
                return -1;
            }
    }
    decode_cfg_t cfg = {&g, order, n_order, T, rule, msg_fmt, w_scale, w_offset, early_every};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > K) nthreads = K > 0 ? K : 1;
    worker_t *ws = (worker_t *)calloc((size_t)nthreads, sizeof(worker_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!ws || !th) {
        free(ws); free(th); free(ord); graph_free(&g);
        return -2;
    }
    const int n = nb * Z, m = mb * Z;
    for (int i = 0; i < nthreads; ++i) {
        ws[i] = (worker_t){&cfg, K, n, m, llr_ch, syn, hard, llr_post, ok, iters_used, i, nthreads, 0};
    }
    int started = 0;
    for (int i = 1; i < nthreads; ++i) {
        if (pthread_create(&th[i], NULL, worker_main, &ws[i]) != 0) break;
        started = i;
    }
    worker_main(&ws[0]);
    /* any worker that failed to start: run its frames here */
    for (int i = started + 1; i < nthreads; ++i) worker_main(&ws[i]);
    for (int i = 1; i <= started; ++i) pthread_join(th[i], NULL);
    int rc = 0;
    for (int i = 0; i < nthreads; ++i)
        if (ws[i].status) rc = ws[i].status;
    free(ws); free(th); free(ord); graph_free(&g);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Learned offset/scaled min-sum: loss and gradient (not part of the      */
/* paper's method; the training target of the learned variant).           */
/*                                                                        */
/* Check rule (for the edge e that receives the message):                  */
/*   r_e = (-1)^{s_m} prod_{k != e} sgn(q_k) * min(max(a_e, 0), 30),      */
/*   a_e = w_scale[t][l][type_e] * min_{k != e} |q_k| - w_offset[t][l][type_e]
/* The rest of the layered update is Methods step 3.  Loss: the mean over   */
/* iterations t and variables n of the binary cross-entropy of the bit     */
/* estimate sigma(-L_qn^(t)) against the transmitted bit x_n,               */
/*   loss = 1/(T n) sum_t sum_n softplus(-(1 - 2 x_n) L_qn^(t)),            */
/* where L^(t) is the posterior after iteration t.  The gradient with      */
/* respect to the weights comes from reverse-mode differentiation of the   */
/* unrolled decoder, written out below (adjoints gL of L_qn and gR of the  */
/* stored L_rmn).                                                          */

static double softplus(double z)
{
    return z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
}

static double sigmoid(double z)
{
    return z >= 0.0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z));
}

/* Min-sum quantities of one check for the edge j: sign, min over the others,
 * argmin index among the others. */
static void minsum_parts(int d, const double *q, int j, double *sign, double *mn, int *arg)
{
    double sg = 1.0, m = INFINITY;
    int a = -1;
    for (int k = 0; k < d; ++k) {
        if (k == j) continue;
        sg *= sgn(q[k]);
        double v = fabs(q[k]);
        if (v < m) {
            m = v;
            a = k;
        }
    }
    if (d == 1) m = ORACLE_CLIP_MAX;
    *sign = sg;
    *mn = m;
    *arg = a;
}

static int train_frame(const graph_t *g, int T, const float *llr_ch, const uint8_t *syn,
                       const uint8_t *x, const double *ws, const double *wo, double *loss,
                       double *gs, double *go)
{
    const int Z = g->Z, mb = g->mb;
    const int n = g->nb * Z;
    const size_t E = (size_t)g->n_circ * (size_t)Z;
    double *Lq = (double *)malloc(sizeof(double) * (size_t)n);
    double *Lr = (double *)calloc(E ? E : 1, sizeof(double));
    double *qh = (double *)malloc(sizeof(double) * (E ? E : 1) * (size_t)(T ? T : 1));   /* q per (t, edge) */
    double *Lh = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(T ? T : 1));     /* L after iteration t */
    double *gL = (double *)calloc((size_t)n, sizeof(double));
    double *gR = (double *)calloc(E ? E : 1, sizeof(double));
    int dmax = g->max_deg > 0 ? g->max_deg : 1;
    double *q = (double *)malloc(sizeof(double) * dmax), *gr = (double *)malloc(sizeof(double) * dmax);
    double *gq = (double *)malloc(sizeof(double) * dmax);
    int *v = (int *)malloc(sizeof(int) * dmax);
    if (!Lq || !Lr || !qh || !Lh || !gL || !gR || !q || !gr || !gq || !v) {
        free(Lq); free(Lr); free(qh); free(Lh); free(gL); free(gR); free(q); free(gr); free(gq); free(v);
        return -2;
    }
    for (int i = 0; i < n; ++i) Lq[i] = (double)llr_ch[i];
    /* forward, recording q and the posteriors after every iteration */
    double lsum = 0.0;
    for (int t = 0; t < T; ++t) {
        for (int l = 0; l < mb; ++l) {
            const int c0 = g->row_first[l], d = g->row_first[l + 1] - c0;
            for (int i = 0; i < Z; ++i) {
                for (int j = 0; j < d; ++j) {
                    const int k = c0 + j;
                    v[j] = g->circ_col[k] * Z + (i + g->circ_shift[k]) % Z;
                    q[j] = Lq[v[j]] - Lr[(size_t)k * Z + i];
                    qh[(size_t)t * E + (size_t)k * Z + i] = q[j];
                }
                const double ssign = (syn[l * Z + i] & 1) ? -1.0 : 1.0;
                for (int j = 0; j < d; ++j) {
                    const int k = c0 + j;
                    double sg, mn;
                    int arg;
                    minsum_parts(d, q, j, &sg, &mn, &arg);
                    const size_t wi = ((size_t)t * mb + l) * 2 + g->circ_type[k];
                    double a = ws[wi] * mn - wo[wi];
                    const double mag = a <= 0.0 ? 0.0 : (a >= ORACLE_CLIP_MAX ? ORACLE_CLIP_MAX : a);
                    const double r = ssign * sg * mag;
                    Lr[(size_t)k * Z + i] = r;
                    Lq[v[j]] = q[j] + r;
                }
            }
        }
        for (int i = 0; i < n; ++i) {
            Lh[(size_t)t * n + i] = Lq[i];
            lsum += softplus(-(1.0 - 2.0 * x[i]) * Lq[i]);
        }
    }
    *loss = T > 0 ? lsum / ((double)T * n) : 0.0;
    /* backward */
    const double scale = T > 0 ? 1.0 / ((double)T * n) : 0.0;
    for (int t = T - 1; t >= 0; --t) {
        /* loss term of the posteriors after iteration t */
        for (int i = 0; i < n; ++i) {
            const double sgx = 1.0 - 2.0 * x[i];
            gL[i] += scale * (-sgx) * sigmoid(-sgx * Lh[(size_t)t * n + i]);
        }
        for (int l = mb - 1; l >= 0; --l) {
            const int c0 = g->row_first[l], d = g->row_first[l + 1] - c0;
            for (int i = 0; i < Z; ++i) {
                for (int j = 0; j < d; ++j) {
                    const int k = c0 + j;
                    v[j] = g->circ_col[k] * Z + (i + g->circ_shift[k]) % Z;
                    q[j] = qh[(size_t)t * E + (size_t)k * Z + i];
                }
                const double ssign = (syn[l * Z + i] & 1) ? -1.0 : 1.0;
                /* adjoint of each new message: it enters L_qn and the stored L_rmn */
                for (int j = 0; j < d; ++j) {
                    gr[j] = gL[v[j]] + gR[(size_t)(c0 + j) * Z + i];
                    gq[j] = gL[v[j]];          /* L_qn = q + r */
                }
                for (int j = 0; j < d; ++j) {
                    const int k = c0 + j;
                    double sg, mn;
                    int arg;
                    minsum_parts(d, q, j, &sg, &mn, &arg);
                    const size_t wi = ((size_t)t * mb + l) * 2 + g->circ_type[k];
                    const double a = ws[wi] * mn - wo[wi];
                    /* outside (0, 30) the clip holds |r| constant: no gradient */
                    if (a <= 0.0 || a >= ORACLE_CLIP_MAX) continue;
                    const double s = ssign * sg;
                    gs[wi] += gr[j] * s * mn;
                    go[wi] += -gr[j] * s;
                    if (arg >= 0) gq[arg] += gr[j] * s * ws[wi] * sgn(q[arg]);
                }
                /* q = L_qn(before) - L_rmn(old) */
                for (int j = 0; j < d; ++j) {
                    gL[v[j]] = gq[j];
                    gR[(size_t)(c0 + j) * Z + i] = -gq[j];
                }
            }
        }
    }
    free(Lq); free(Lr); free(qh); free(Lh); free(gL); free(gR); free(q); free(gr); free(gq); free(v);
    return 0;
}

/*
 * Learned min-sum training quantities for K frames (base-row order):
 *   x          : [K][n] transmitted bits
 *   w_scale, w_offset : [T][mb][2] weights (type 0: edge to a variable of
 *                degree > 1, type 1: edge to a degree-1 variable)
 *   loss       : [K] out, per-frame loss
 *   g_scale, g_offset : [T][mb][2] out, gradient of the SUM of the K losses
 * Returns 0, or <0 on invalid input / allocation failure.
 */
int oracle_minsum_train(int mb, int nb, int Z, const int8_t *base, const int32_t *shifts, int K,
                        int T, const float *llr_ch, const uint8_t *syn, const uint8_t *x,
                        const double *w_scale, const double *w_offset, double *loss,
                        double *g_scale, double *g_offset)
{
    if (K < 0 || T < 0 || !base || !shifts || !w_scale || !w_offset || !g_scale || !g_offset)
        return -1;
    graph_t g;
    int st = graph_build(mb, nb, Z, base, shifts, &g);
    if (st) return st;
    const size_t nw = (size_t)T * mb * 2;
    for (size_t i = 0; i < nw; ++i) g_scale[i] = g_offset[i] = 0.0;
    const int n = nb * Z, m = mb * Z;
    int rc = 0;
    for (int k = 0; k < K && !rc; ++k)
        rc = train_frame(&g, T, llr_ch + (size_t)k * n, syn + (size_t)k * m, x + (size_t)k * n,
                         w_scale, w_offset, loss + k, g_scale, g_offset);
    graph_free(&g);
    return rc;
}
