/*
 * FP64 CPU oracle for belief-propagation (BP) decoding of LDPC codes over
 * GF(q), q = 2^p <= 256, under the parallel (PUS) and the sequential (SUS)
 * updating schedules, with optional dynamical Markov block priors.
 *
 * Paper: N. Yacov, H. Efraim, H. Kfir, I. Kanter, O. Shental, "Parallel vs.
 * Sequential Belief Propagation Decoding of LDPC Codes over GF(q) and Markov
 * Sources" (arXiv cs/0605069).  Section and equation numbers below are the
 * paper's.
 *
 * TEST INFRASTRUCTURE.  This file is the slow, literal reference that the
 * CUDA decoder is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg load it.  It shares no code, header or
 * table with the CUDA library.
 *
 * Everything is computed in double precision, literally in the paper's order:
 *   channel likelihoods and priors p_j (Sec. 2, BSC initialisation formula
 *     and the footnote on other channels; priors of Sec. 2),
 *   q_ij <- p_j initialisation (Sec. 2, noise-bit initialisation),
 *   horizontal pass r_ij (Eq. 3) as the configuration sum regrouped into
 *     successive XOR-convolutions (distributivity; no transform),
 *   vertical pass q_ij (Eq. 4), pseudo-posterior Q_j (Eq. 5),
 *   hard decision by clipping Q_j and the test H x = z (Sec. 2),
 *   PUS: all r from the previous q, then all q (Sec. 2);
 *   SUS: per column j in order, r_ij for all checks of j, then q_ij for j,
 *     and Q after the sweep (Sec. 2, SUS steps 1-4),
 *   Markov prior P_i (Eq. 6 as a double sum; Eq. 7 as a separate routine).
 *
 * Readings where the paper is silent (each is stated where it is used):
 *   R1 field: GF(2^p) built from a primitive polynomial (parameter);
 *   R2 symbol bits: bit k of a is (a >> k) & 1; BPSK maps bit 0 to +1;
 *   R3 r is normalised to sum 1 (q and Q do not change in exact arithmetic);
 *   R4 a vector whose sum is 0 is replaced by the uniform vector (counted);
 *   R5 hard decision = argmax, lowest symbol on ties;
 *   R6 the test runs after every iteration, so the count is >= 1;
 *   R7 Markov prior: Jacobi (all P from the finished iteration's Q),
 *      boundaries P_0 = pi_b * sum_c M_bc Q_1^c and
 *      P_{K-1} = sum_a Q_{K-2}^a M_ab, initial P = pi (stationary);
 *      transition rows renormalised.
 *   R8 in SUS, Q_j uses the r_ij computed at column j's step.
 *   R9 Markov prior inside SUS, Gauss-Seidel (markov = 2; a variant the
 *      paper leaves open): P_i is re-estimated by Eq. 6 just before the
 *      sweep reaches source symbol i's column, from the pseudo-posteriors of
 *      its neighbours as they stand (this sweep's where the sweep has already
 *      passed them, the previous sweep's otherwise); before a symbol's first
 *      visit its pseudo-posterior is its initial belief p_j (channel
 *      likelihood times pi, normalised).  No update between sweeps.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

/* ---------------------------------------------------------------- GF(2^p) */
/* R1: exp/log tables of a primitive element x; the polynomial must be primitive. */
typedef struct {
    int q, p;
    int ex[512];
    int lg[256];
} ogf;

static unsigned default_poly(int p) {
    switch (p) {
    case 1: return 0x3;   /* x + 1 */
    case 2: return 0x7;   /* x^2 + x + 1 */
    case 3: return 0xB;   /* x^3 + x + 1 */
    case 4: return 0x13;  /* x^4 + x + 1 */
    case 5: return 0x25;  /* x^5 + x^2 + 1 */
    case 6: return 0x43;  /* x^6 + x + 1 */
    case 7: return 0x89;  /* x^7 + x^3 + 1 */
    case 8: return 0x11D; /* x^8 + x^4 + x^3 + x^2 + 1 */
    }
    return 0;
}

static int ilog2q(int q) {
    int p = 0;
    while ((1 << p) < q) p++;
    return ((1 << p) == q && p >= 1 && p <= 8) ? p : -1;
}

static int ogf_init(ogf* g, int q, unsigned poly) {
    int p = ilog2q(q);
    if (p < 0) return OR_EINVAL;
    if (poly == 0) poly = default_poly(p);
    if ((poly >> p) != 1u) return OR_EINVAL; /* degree must be p */
    g->q = q;
    g->p = p;
    for (int a = 0; a < 256; a++) g->lg[a] = -1;
    int v = 1;
    for (int i = 0; i < q - 1; i++) {
        if (g->lg[v] != -1) return OR_EINVAL; /* x has order < q-1: not primitive */
        g->ex[i] = v;
        g->lg[v] = i;
        v <<= 1;
        if (v & q) v ^= (int)poly;
    }
    if (v != 1) return OR_EINVAL;
    for (int i = q - 1; i < 512; i++) g->ex[i] = g->ex[i % (q - 1)];
    return OR_OK;
}

static inline int gf_mul(const ogf* g, int a, int b) {
    if (a == 0 || b == 0) return 0;
    return g->ex[g->lg[a] + g->lg[b]];
}

static inline int gf_inv(const ogf* g, int a) { return g->ex[(g->q - 1 - g->lg[a]) % (g->q - 1)]; }

/* ------------------------------------------------------------- code graph */
typedef struct {
    int q, M, N;
    long E;
    int* rp;  /* [M+1] row pointer; edges sorted by (row, col) */
    int* er;  /* [E] row of edge */
    int* ec;  /* [E] column of edge */
    int* eh;  /* [E] GF value of edge */
    int* cp;  /* [N+1] column pointer */
    int* ce;  /* [E] edge ids of each column, rows increasing */
    int dcmax, dvmax;
} ocode;

static void ocode_free(ocode* c) {
    free(c->rp); free(c->er); free(c->ec); free(c->eh); free(c->cp); free(c->ce);
    memset(c, 0, sizeof(*c));
}

static int ocode_build(ocode* c, int q, int M, int N, long E, const int32_t* row, const int32_t* col,
                       const int32_t* val) {
    memset(c, 0, sizeof(*c));
    c->q = q; c->M = M; c->N = N; c->E = E;
    c->rp = calloc((size_t)M + 1, sizeof(int));
    c->cp = calloc((size_t)N + 1, sizeof(int));
    c->er = malloc(sizeof(int) * (size_t)(E ? E : 1));
    c->ec = malloc(sizeof(int) * (size_t)(E ? E : 1));
    c->eh = malloc(sizeof(int) * (size_t)(E ? E : 1));
    c->ce = malloc(sizeof(int) * (size_t)(E ? E : 1));
    if (!c->rp || !c->cp || !c->er || !c->ec || !c->eh || !c->ce) { ocode_free(c); return OR_ENOMEM; }
    for (long e = 0; e < E; e++) {
        if (row[e] < 0 || row[e] >= M || col[e] < 0 || col[e] >= N || val[e] <= 0 || val[e] >= q) {
            ocode_free(c); return OR_EINVAL;
        }
        if (e > 0 && (row[e] < row[e - 1] || (row[e] == row[e - 1] && col[e] <= col[e - 1]))) {
            ocode_free(c); return OR_EINVAL; /* must be sorted by (row, col) without duplicates */
        }
        c->er[e] = row[e]; c->ec[e] = col[e]; c->eh[e] = val[e];
        c->rp[row[e] + 1]++;
        c->cp[col[e] + 1]++;
    }
    for (int i = 0; i < M; i++) c->rp[i + 1] += c->rp[i];
    for (int j = 0; j < N; j++) c->cp[j + 1] += c->cp[j];
    int* fill = calloc((size_t)N + 1, sizeof(int));
    if (!fill) { ocode_free(c); return OR_ENOMEM; }
    for (long e = 0; e < E; e++) { int j = c->ec[e]; c->ce[c->cp[j] + fill[j]++] = (int)e; }
    free(fill);
    for (int i = 0; i < M; i++) if (c->rp[i + 1] - c->rp[i] > c->dcmax) c->dcmax = c->rp[i + 1] - c->rp[i];
    for (int j = 0; j < N; j++) if (c->cp[j + 1] - c->cp[j] > c->dvmax) c->dvmax = c->cp[j + 1] - c->cp[j];
    return OR_OK;
}

/* ----------------------------------------------------------- vector utils */
/* R3/R4: scale to sum 1; a zero (or non-finite) sum gives the uniform vector. */
static int normalise(double* v, int q) {
    double s = 0.0;
    for (int a = 0; a < q; a++) s += v[a];
    if (!(s > 0.0) || !isfinite(s)) {
        for (int a = 0; a < q; a++) v[a] = 1.0 / q;
        return 1;
    }
    for (int a = 0; a < q; a++) v[a] /= s;
    return 0;
}

/* R5: clipping Q_j to a symbol = argmax, lowest index on ties. */
static int argmax_low(const double* v, int q) {
    int b = 0;
    for (int a = 1; a < q; a++) if (v[a] > v[b]) b = a;
    return b;
}

/* ------------------------------------------------------ channel (Sec. 2) */
enum { CH_BSC = 0, CH_BEC = 1, CH_BIAWGN = 2, CH_LOGLIK = 3 };

/* Likelihood of every symbol a given the observation of its p bits.
 * BSC (Sec. 2): f^L (1-f)^(p-L) with L the number of bits where a and the
 *   received word differ (the paper's formula is the case of a received 0).
 * BEC: 1 for symbols that agree with every non-erased bit (value 2 = erased).
 * BI-AWGN, BPSK bit 0 -> +1 (R2): exp(-sum_k (y_k - s_k(a))^2 / (2 sigma^2)),
 *   formed in the log domain and shifted by its maximum.
 * LOGLIK: the observation holds q log-likelihoods.
 * A punctured symbol has no observation: uniform. */
static void channel_likelihood(int kind, double param, int q, int p, const float* y, int punctured, double* L) {
    if (punctured) {
        for (int a = 0; a < q; a++) L[a] = 1.0;
    } else if (kind == CH_BSC) {
        for (int a = 0; a < q; a++) {
            double v = 1.0;
            for (int k = 0; k < p; k++) {
                int bit = (a >> k) & 1;
                int rx = y[k] > 0.5f ? 1 : 0;
                v *= (bit == rx) ? (1.0 - param) : param;
            }
            L[a] = v;
        }
    } else if (kind == CH_BEC) {
        for (int a = 0; a < q; a++) {
            double v = 1.0;
            for (int k = 0; k < p; k++) {
                if (y[k] > 1.5f) continue; /* erased */
                int bit = (a >> k) & 1;
                int rx = y[k] > 0.5f ? 1 : 0;
                if (bit != rx) v = 0.0;
            }
            L[a] = v;
        }
    } else if (kind == CH_BIAWGN) {
        double mx = -INFINITY;
        for (int a = 0; a < q; a++) {
            double ll = 0.0;
            for (int k = 0; k < p; k++) {
                double s = ((a >> k) & 1) ? -1.0 : 1.0;
                double d = (double)y[k] - s;
                ll -= d * d / (2.0 * param * param);
            }
            L[a] = ll;
            if (ll > mx) mx = ll;
        }
        for (int a = 0; a < q; a++) L[a] = exp(L[a] - mx);
    } else { /* CH_LOGLIK */
        double mx = -INFINITY;
        for (int a = 0; a < q; a++) if ((double)y[a] > mx) mx = (double)y[a];
        for (int a = 0; a < q; a++) L[a] = exp((double)y[a] - mx);
    }
    normalise(L, q);
}

/* --------------------------------------------------- horizontal pass Eq. 3 */
/* r_ij^a for the k-th edge of check i (degree d, GF values h[0..d-1],
 * incoming q vectors qv[0..d-1], syndrome value z):
 *   r^a = sum over the symbols x_m of the other edges with
 *         h_k a + sum_{m != k} h_m x_m = z   of   prod_{m != k} q_m^{x_m}.
 * Addition in GF(2^p) is XOR.  The configuration sum is regrouped by
 * distributivity into successive sums: u is the distribution (unnormalised)
 * of y = sum_{m != k} h_m x_m, grown one edge at a time; then
 * r^a = u[z + h_k a]. */
static void check_edge_direct(const ogf* g, int d, const int* h, const double* const* qv, int k, int z,
                              double* r, double* u, double* v) {
    int q = g->q;
    for (int y = 0; y < q; y++) u[y] = 0.0;
    u[0] = 1.0; /* empty sum: y = 0 with weight 1 */
    for (int m = 0; m < d; m++) {
        if (m == k) continue;
        for (int y = 0; y < q; y++) v[y] = 0.0;
        for (int y = 0; y < q; y++) {
            if (u[y] == 0.0) continue;
            for (int x = 0; x < q; x++) v[y ^ gf_mul(g, h[m], x)] += u[y] * qv[m][x];
        }
        for (int y = 0; y < q; y++) u[y] = v[y];
    }
    for (int a = 0; a < q; a++) r[a] = u[z ^ gf_mul(g, h[k], a)];
}

/* Textbook fast Walsh-Hadamard transform (unnormalised), in place. */
static void fwht(double* x, int q) {
    for (int len = 1; len < q; len <<= 1)
        for (int i = 0; i < q; i += len << 1)
            for (int j = i; j < i + len; j++) {
                double a = x[j], b = x[j + len];
                x[j] = a + b;
                x[j + len] = a - b;
            }
}

/* The same r as check_edge_direct, through the convolution theorem for
 * XOR-convolution: the distribution of h_m x_m is q_m relabelled by
 * b = h_m x; transform, multiply the other edges' transforms, transform back
 * and divide by q.  Rounding can leave tiny negatives: they are set to 0. */
static void check_edge_wht(const ogf* g, int d, const int* h, const double* const* qv, int k, int z,
                           double* r, double* u, double* v) {
    int q = g->q;
    for (int w = 0; w < q; w++) u[w] = 1.0;
    for (int m = 0; m < d; m++) {
        if (m == k) continue;
        for (int b = 0; b < q; b++) v[b] = 0.0;
        for (int x = 0; x < q; x++) v[gf_mul(g, h[m], x)] = qv[m][x];
        fwht(v, q);
        for (int w = 0; w < q; w++) u[w] *= v[w];
    }
    fwht(u, q);
    for (int y = 0; y < q; y++) u[y] = u[y] / q > 0.0 ? u[y] / q : 0.0;
    for (int a = 0; a < q; a++) r[a] = u[z ^ gf_mul(g, h[k], a)];
}

/* -------------------------------------------------- Markov prior Eqs. 6-7 */
/* Stationary distribution pi of the row-stochastic matrix T (pi T = pi,
 * sum pi = 1) by Gaussian elimination with partial pivoting. */
static int stationary(const double* T, int q, double* pi) {
    double* A = malloc(sizeof(double) * (size_t)q * (size_t)(q + 1));
    if (!A) return OR_ENOMEM;
    /* rows 0..q-2: (T^T - I) pi = 0 ; last row: sum pi = 1 */
    for (int r = 0; r < q; r++) {
        for (int c = 0; c < q; c++) A[r * (q + 1) + c] = (r == q - 1) ? 1.0 : T[c * q + r] - (r == c ? 1.0 : 0.0);
        A[r * (q + 1) + q] = (r == q - 1) ? 1.0 : 0.0;
    }
    for (int c = 0; c < q; c++) {
        int piv = c;
        for (int r = c + 1; r < q; r++) if (fabs(A[r * (q + 1) + c]) > fabs(A[piv * (q + 1) + c])) piv = r;
        if (fabs(A[piv * (q + 1) + c]) < 1e-300) { free(A); return OR_EINVAL; }
        if (piv != c)
            for (int k = 0; k <= q; k++) { double t = A[c * (q + 1) + k]; A[c * (q + 1) + k] = A[piv * (q + 1) + k]; A[piv * (q + 1) + k] = t; }
        for (int r = 0; r < q; r++) {
            if (r == c) continue;
            double f = A[r * (q + 1) + c] / A[c * (q + 1) + c];
            if (f == 0.0) continue;
            for (int k = c; k <= q; k++) A[r * (q + 1) + k] -= f * A[c * (q + 1) + k];
        }
    }
    for (int r = 0; r < q; r++) pi[r] = A[r * (q + 1) + q] / A[r * (q + 1) + r];
    free(A);
    return OR_OK;
}

/* Eq. 6 for source position i of K, with Qm = Q_{i-1} and Qp = Q_{i+1}
 * (NULL at the ends, R7):
 *   P_i^b = sum_{a,c} Q_{i-1}^a M_ab M_bc Q_{i+1}^c,
 * at i = 0: pi_b sum_c M_bc Q_1^c; at i = K-1: sum_a Q_{K-2}^a M_ab;
 * K = 1: pi_b.  Normalised. */
static void markov_prior_eq6(const double* Mt, const double* pi, int q, const double* Qm, const double* Qp, double* P) {
    for (int b = 0; b < q; b++) {
        double s = 0.0;
        if (Qm && Qp) {
            for (int a = 0; a < q; a++)
                for (int c = 0; c < q; c++) s += Qm[a] * Mt[a * q + b] * Mt[b * q + c] * Qp[c];
        } else if (Qp) {
            for (int c = 0; c < q; c++) s += pi[b] * Mt[b * q + c] * Qp[c];
        } else if (Qm) {
            for (int a = 0; a < q; a++) s += Qm[a] * Mt[a * q + b];
        } else {
            s = pi[b];
        }
        P[b] = s;
    }
    normalise(P, q);
}

/* Eq. 7: the same quantity with the double sum factored,
 *   P_i^b = (sum_a Q_{i-1}^a M_ab) (sum_c M_bc Q_{i+1}^c). */
static void markov_prior_eq7(const double* Mt, const double* pi, int q, const double* Qm, const double* Qp, double* P) {
    for (int b = 0; b < q; b++) {
        double left = 0.0, right = 0.0;
        if (Qm) { for (int a = 0; a < q; a++) left += Qm[a] * Mt[a * q + b]; }
        else left = pi[b];
        if (Qp) { for (int c = 0; c < q; c++) right += Mt[b * q + c] * Qp[c]; }
        else right = 1.0;
        P[b] = left * right;
    }
    normalise(P, q);
}

/* ------------------------------------------------------------- decoder */
typedef struct {
    const ogf* g;
    const ocode* c;
    int kind;
    double param;          /* f, eps or sigma */
    int schedule;          /* 0 PUS, 1 SUS */
    int use_wht;           /* 0: direct configuration sum, 1: transform route */
    int markov;            /* 0 iid, 1 Markov block priors */
    int gs;                /* Markov priors re-estimated inside the SUS sweep (R9) */
    int round32;           /* conditioning probe: store every message rounded to float */
    const double* Mt;      /* [q*q] row-normalised transition matrix */
    const double* pi;      /* [q] */
    int K;                 /* number of source positions */
    const int* src_pos;    /* [K] ordered source positions */
    const int* src_index;  /* [N] position -> index in src_pos, or -1 */
} odec;

typedef struct {
    double* L;    /* [N][q] channel likelihoods */
    double* P;    /* [K][q] source priors */
    double* pj;   /* [q] scratch prior of the current symbol */
    double* qm;   /* [E][q] q_ij messages */
    double* rm;   /* [E][q] r_ij messages */
    double* Q;    /* [N][q] pseudo-posteriors */
    double* u;
    double* v;
    double** qv;  /* [dcmax] */
    int* h;       /* [dcmax] */
    int* xh;      /* [N] */
    long zero_sums;
} owork;

/* The conditioning probe (not the decoder's arithmetic; round32 != 0): a
 * message stored rounded to the nearest float, as a decoder that keeps FP32
 * messages does.  With round32 = k >= 2 every channel likelihood is also moved
 * by one float ulp up, down or not at all, by a hash of (k, frame, symbol,
 * entry): one of the FP32 roundings a decoder computing them could meet. */
static void store32(const odec* D, double* v, int q) {
    if (D->round32)
        for (int a = 0; a < q; a++) v[a] = (double)(float)v[a];
}

/* p_j = L_j * P_j, normalised (Sec. 2 priors; i.i.d. source: uniform, no effect). */
static void prior_of(const odec* D, const owork* W, int j, double* out) {
    int q = D->g->q;
    const double* L = W->L + (size_t)j * q;
    int si = D->markov ? D->src_index[j] : -1;
    for (int a = 0; a < q; a++) out[a] = L[a] * (si >= 0 ? W->P[(size_t)si * q + a] : 1.0);
    normalise(out, q);
}

/* r for every edge of check i from the current q messages (Eq. 3). */
static void horizontal_check(const odec* D, owork* W, int i, int z_i, int only_edge) {
    const ocode* c = D->c;
    int q = c->q;
    int e0 = c->rp[i], d = c->rp[i + 1] - c->rp[i];
    for (int m = 0; m < d; m++) { W->h[m] = c->eh[e0 + m]; W->qv[m] = W->qm + (size_t)(e0 + m) * q; }
    for (int k = 0; k < d; k++) {
        if (only_edge >= 0 && e0 + k != only_edge) continue;
        double* r = W->rm + (size_t)(e0 + k) * q;
        if (D->use_wht) check_edge_wht(D->g, d, W->h, (const double* const*)W->qv, k, z_i, r, W->u, W->v);
        else check_edge_direct(D->g, d, W->h, (const double* const*)W->qv, k, z_i, r, W->u, W->v);
        W->zero_sums += normalise(r, q);
        store32(D, r, q);
    }
}

/* Vertical pass for column j (Eq. 4) and its pseudo-posterior (Eq. 5). */
static void vertical_column(const odec* D, owork* W, int j) {
    const ocode* c = D->c;
    int q = c->q;
    prior_of(D, W, j, W->pj);
    int b0 = c->cp[j], dv = c->cp[j + 1] - c->cp[j];
    for (int k = 0; k < dv; k++) {
        double* qo = W->qm + (size_t)c->ce[b0 + k] * q;
        for (int a = 0; a < q; a++) {
            double v = W->pj[a];
            for (int m = 0; m < dv; m++) if (m != k) v *= W->rm[(size_t)c->ce[b0 + m] * q + a];
            qo[a] = v;
        }
        W->zero_sums += normalise(qo, q);
        store32(D, qo, q);
    }
    double* Qj = W->Q + (size_t)j * q;
    for (int a = 0; a < q; a++) {
        double v = W->pj[a];
        for (int m = 0; m < dv; m++) v *= W->rm[(size_t)c->ce[b0 + m] * q + a];
        Qj[a] = v;
    }
    W->zero_sums += normalise(Qj, q);
    store32(D, Qj, q);
}

/* One iteration of the chosen schedule, ending with Q for every symbol. */
static void one_iteration(const odec* D, owork* W, const uint8_t* z) {
    const ocode* c = D->c;
    if (D->schedule == 0) {
        /* PUS: horizontal pass over all checks (every r from the previous
         * iteration's q), then the vertical pass over all columns. */
        for (int i = 0; i < c->M; i++) horizontal_check(D, W, i, z ? z[i] : 0, -1);
        for (int j = 0; j < c->N; j++) vertical_column(D, W, j);
    } else {
        /* SUS: for each column j in order: step 1, r_ij for every check i of
         * column j from the current q; step 2, q_ij for column j; step 3,
         * next column; step 4, Q (computed with column j, R8). */
        for (int j = 0; j < c->N; j++) {
            if (D->gs && D->src_index[j] >= 0) {   /* R9: P_i as the sweep reaches i */
                int q = c->q, i = D->src_index[j], K = D->K;
                const double* Qm = i > 0 ? W->Q + (size_t)D->src_pos[i - 1] * q : NULL;
                const double* Qp = i < K - 1 ? W->Q + (size_t)D->src_pos[i + 1] * q : NULL;
                markov_prior_eq6(D->Mt, D->pi, q, Qm, Qp, W->P + (size_t)i * q);
            }
            for (int k = c->cp[j]; k < c->cp[j + 1]; k++) {
                int e = c->ce[k];
                int i = c->er[e];
                horizontal_check(D, W, i, z ? z[i] : 0, e);
            }
            vertical_column(D, W, j);
        }
    }
}

/* Clip every Q_j and test H x = z; returns 1 when all M equations hold. */
static int harden_and_test(const odec* D, owork* W, const uint8_t* z) {
    const ocode* c = D->c;
    int q = c->q;
    for (int j = 0; j < c->N; j++) W->xh[j] = argmax_low(W->Q + (size_t)j * q, q);
    for (int i = 0; i < c->M; i++) {
        int s = 0;
        for (int e = c->rp[i]; e < c->rp[i + 1]; e++) s ^= gf_mul(D->g, c->eh[e], W->xh[c->ec[e]]);
        if (s != (z ? z[i] : 0)) return 0;
    }
    return 1;
}

/* Dynamical block priors after an iteration (Eq. 6, Jacobi reading R7). */
static void update_priors(const odec* D, owork* W, double* Pout) {
    int q = D->g->q, K = D->K;
    for (int i = 0; i < K; i++) {
        const double* Qm = i > 0 ? W->Q + (size_t)D->src_pos[i - 1] * q : NULL;
        const double* Qp = i < K - 1 ? W->Q + (size_t)D->src_pos[i + 1] * q : NULL;
        markov_prior_eq6(D->Mt, D->pi, q, Qm, Qp, Pout + (size_t)i * q);
    }
}

static int owork_alloc(owork* W, const ocode* c, int K) {
    int q = c->q;
    memset(W, 0, sizeof(*W));
    W->L = malloc(sizeof(double) * (size_t)c->N * q);
    W->P = malloc(sizeof(double) * (size_t)(K > 0 ? K : 1) * q);
    W->pj = malloc(sizeof(double) * q);
    W->qm = malloc(sizeof(double) * (size_t)(c->E ? c->E : 1) * q);
    W->rm = malloc(sizeof(double) * (size_t)(c->E ? c->E : 1) * q);
    W->Q = malloc(sizeof(double) * (size_t)c->N * q);
    W->u = malloc(sizeof(double) * q);
    W->v = malloc(sizeof(double) * q);
    W->qv = malloc(sizeof(double*) * (size_t)(c->dcmax + 1));
    W->h = malloc(sizeof(int) * (size_t)(c->dcmax + 1));
    W->xh = malloc(sizeof(int) * (size_t)(c->N + 1));
    if (!W->L || !W->P || !W->pj || !W->qm || !W->rm || !W->Q || !W->u || !W->v || !W->qv || !W->h || !W->xh)
        return OR_ENOMEM;
    return OR_OK;
}

static void owork_free(owork* W) {
    free(W->L); free(W->P); free(W->pj); free(W->qm); free(W->rm); free(W->Q);
    free(W->u); free(W->v); free(W->qv); free(W->h); free(W->xh);
}

typedef struct {
    int q; unsigned poly; int M, N; long E;
    const int32_t *row, *col, *val;
    int n_frames;
    int kind;
    const double* param;      /* [F] channel parameter per frame */
    const float* obs;         /* [F][N][p] or [F][N][q] (LOGLIK) */
    const uint8_t* punct;     /* [N] or NULL */
    const uint8_t* syn;       /* [F][M] or NULL */
    int schedule, use_wht, early_stop, max_iter;
    int markov; const double* T; int K; const int32_t* src_pos;
    int n_threads;
    int round32;              /* conditioning probe (store32) */
} oargs;

typedef struct {
    ogf g;
    ocode c;
    double* Mt;
    double pi[256];
    int* src_pos;
    int* src_index;
} oshared;

static void oshared_free(oshared* S) {
    ocode_free(&S->c);
    free(S->Mt); free(S->src_pos); free(S->src_index);
}

static int oshared_init(oshared* S, const oargs* A) {
    memset(S, 0, sizeof(*S));
    if (A->max_iter < 1 || A->n_frames < 0 || A->kind < 0 || A->kind > 3) return OR_EINVAL;
    int rc = ogf_init(&S->g, A->q, A->poly);
    if (rc) return rc;
    rc = ocode_build(&S->c, A->q, A->M, A->N, A->E, A->row, A->col, A->val);
    if (rc) return rc;
    int q = A->q;
    S->src_index = malloc(sizeof(int) * (size_t)(A->N + 1));
    S->src_pos = malloc(sizeof(int) * (size_t)(A->K + 1));
    S->Mt = malloc(sizeof(double) * (size_t)q * q);
    if (!S->src_index || !S->src_pos || !S->Mt) { oshared_free(S); return OR_ENOMEM; }
    for (int j = 0; j < A->N; j++) S->src_index[j] = -1;
    if (A->markov == 2 && A->schedule != 1) { oshared_free(S); return OR_EINVAL; }   /* R9: SUS only */
    if (A->markov) {
        if (!A->T || A->K < 1 || A->K > A->N) { oshared_free(S); return OR_EINVAL; }
        for (int a = 0; a < q; a++) { /* R7: rows renormalised */
            double s = 0.0;
            for (int b = 0; b < q; b++) { if (!(A->T[a * q + b] >= 0.0)) { oshared_free(S); return OR_EINVAL; } s += A->T[a * q + b]; }
            if (!(s > 0.0)) { oshared_free(S); return OR_EINVAL; }
            for (int b = 0; b < q; b++) S->Mt[a * q + b] = A->T[a * q + b] / s;
        }
        if (stationary(S->Mt, q, S->pi)) { oshared_free(S); return OR_EINVAL; }
        for (int i = 0; i < A->K; i++) {
            int j = A->src_pos ? A->src_pos[i] : i;
            if (j < 0 || j >= A->N || S->src_index[j] != -1) { oshared_free(S); return OR_EINVAL; }
            S->src_pos[i] = j;
            S->src_index[j] = i;
        }
    }
    return OR_OK;
}

static void odec_of(odec* D, const oshared* S, const oargs* A, int f) {
    D->g = &S->g; D->c = &S->c; D->kind = A->kind; D->param = A->param ? A->param[f] : 0.0;
    D->schedule = A->schedule; D->use_wht = A->use_wht; D->markov = A->markov != 0;
    D->gs = A->markov == 2;
    D->round32 = A->round32;
    D->Mt = S->Mt; D->pi = S->pi; D->K = A->markov ? A->K : 0;
    D->src_pos = S->src_pos; D->src_index = S->src_index;
}

/* Channel likelihoods of frame f and the initial priors (pi for source symbols). */
static uint64_t mix64(uint64_t x) {   /* splitmix64 finaliser */
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

static void frame_setup(const odec* D, owork* W, const oargs* A, int f) {
    int q = A->q, p = D->g->p, N = A->N;
    int stride = A->kind == CH_LOGLIK ? q : p;
    for (int j = 0; j < N; j++) {
        double* L = W->L + (size_t)j * q;
        channel_likelihood(A->kind, D->param, q, p, A->obs + ((size_t)f * N + j) * stride,
                           A->punct ? A->punct[j] : 0, L);
        if (D->round32 >= 2)
            for (int a = 0; a < q; a++) {
                const uint64_t h = mix64(((uint64_t)D->round32 << 48) ^ ((uint64_t)f << 32) ^ ((uint64_t)j << 9) ^ a);
                const float x = (float)L[a];
                const int step = (int)(h % 3) - 1;
                L[a] = step == 0 || x == 0.0f ? x : nextafterf(x, step > 0 ? INFINITY : 0.0f);
            }
        else
            store32(D, L, q);
    }
    for (int i = 0; i < D->K; i++)
        for (int a = 0; a < q; a++) W->P[(size_t)i * q + a] = D->pi[a];
}

/*
 * Full decode of n_frames frames.  Outputs: xhat [F][N], iters [F], conv [F],
 * optionally post [F][N][q] (final Q), trace_x [F][max_iter][N] (hard
 * decisions after each iteration; 255 after stopping) and trace_gap
 * [F][max_iter][N] (Q's top-two gap after each iteration), zero_sums [F].
 */
int oracle_decode(int q, unsigned poly, int M, int N, long E, const int32_t* row, const int32_t* col,
                  const int32_t* val, int n_frames, int kind, const double* param, const float* obs,
                  const uint8_t* punct, const uint8_t* syn, int schedule, int use_wht, int early_stop,
                  int max_iter, int markov, const double* T, int K, const int32_t* src_pos, uint8_t* xhat,
                  int32_t* iters, uint8_t* conv, double* post, uint8_t* trace_x, float* trace_gap,
                  int64_t* zero_sums, int n_threads, int round32) {
    oargs A = {q, poly, M, N, E, row, col, val, n_frames, kind, param, obs, punct, syn,
               schedule, use_wht, early_stop, max_iter, markov, T, K, src_pos, n_threads, round32};
    oshared S;
    int rc = oshared_init(&S, &A);
    if (rc) return rc;
    int err = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        owork W;
        int mine = owork_alloc(&W, &S.c, K);
        if (mine) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = mine;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int f = 0; f < n_frames; f++) {
            if (mine) continue;
            odec D;
            odec_of(&D, &S, &A, f);
            W.zero_sums = 0;
            frame_setup(&D, &W, &A, f);
            const uint8_t* z = syn ? syn + (size_t)f * M : NULL;
            /* q_ij <- p_j on every edge of column j (Sec. 2 initialisation). */
            for (int j = 0; j < N; j++) {
                prior_of(&D, &W, j, W.pj);
                for (int k = S.c.cp[j]; k < S.c.cp[j + 1]; k++)
                    memcpy(W.qm + (size_t)S.c.ce[k] * q, W.pj, sizeof(double) * q);
            }
            /* R9: pseudo-posteriors before any visit are the initial beliefs */
            if (D.gs)
                for (int j = 0; j < N; j++) prior_of(&D, &W, j, W.Q + (size_t)j * q);
            int t, ok = 0;
            for (t = 1; t <= max_iter; t++) {
                one_iteration(&D, &W, z);
                ok = harden_and_test(&D, &W, z);
                if (trace_x || trace_gap) {
                    for (int j = 0; j < N; j++) {
                        size_t o = ((size_t)f * max_iter + (t - 1)) * N + j;
                        if (trace_x) trace_x[o] = (uint8_t)W.xh[j];
                        if (trace_gap) {
                            const double* Qj = W.Q + (size_t)j * q;
                            double b1 = -1.0, b2 = -1.0;
                            for (int a = 0; a < q; a++) {
                                if (Qj[a] > b1) { b2 = b1; b1 = Qj[a]; }
                                else if (Qj[a] > b2) b2 = Qj[a];
                            }
                            trace_gap[o] = (float)(b1 - b2);
                        }
                    }
                }
                if (ok && early_stop) break;
                if (t < max_iter && D.markov && !D.gs) {
                    update_priors(&D, &W, W.P);
                }
            }
            if (t > max_iter) t = max_iter;
            if (trace_x)
                for (int t2 = t; t2 < max_iter; t2++)
                    memset(trace_x + ((size_t)f * max_iter + t2) * N, 255, (size_t)N);
            for (int j = 0; j < N; j++) xhat[(size_t)f * N + j] = (uint8_t)W.xh[j];
            iters[f] = t;
            conv[f] = (uint8_t)ok;
            if (post) memcpy(post + (size_t)f * N * q, W.Q, sizeof(double) * (size_t)N * q);
            if (zero_sums) zero_sums[f] = W.zero_sums;
        }
        owork_free(&W);
    }
    oshared_free(&S);
    return err;
}

/*
 * Exactly one iteration from a given state, for lock-step comparison:
 * msg [F][E][q] holds q_ij (edges in (row, col) order) and is overwritten
 * with the q_ij after the iteration; prior [F][K][q] holds the P used in
 * this iteration (Markov only) and prior_out receives Eq. 6 from the new Q.
 * Outputs post [F][N][q], xhat [F][N] and sat [F] (1 when H x = z).
 */
int oracle_step(int q, unsigned poly, int M, int N, long E, const int32_t* row, const int32_t* col,
                const int32_t* val, int n_frames, int kind, const double* param, const float* obs,
                const uint8_t* punct, const uint8_t* syn, int schedule, int use_wht, int markov,
                const double* T, int K, const int32_t* src_pos, double* msg, const double* prior,
                double* prior_out, double* post, uint8_t* xhat, uint8_t* sat, int n_threads) {
    oargs A = {q, poly, M, N, E, row, col, val, n_frames, kind, param, obs, punct, syn,
               schedule, use_wht, 1, 1, markov, T, K, src_pos, n_threads, 0};
    oshared S;
    int rc = oshared_init(&S, &A);
    if (rc) return rc;
    int err = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        owork W;
        int mine = owork_alloc(&W, &S.c, K);
        if (mine) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = mine;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int f = 0; f < n_frames; f++) {
            if (mine) continue;
            odec D;
            odec_of(&D, &S, &A, f);
            frame_setup(&D, &W, &A, f);
            if (D.markov) memcpy(W.P, prior + (size_t)f * K * q, sizeof(double) * (size_t)K * q);
            double* mf = msg + (size_t)f * E * q;
            memcpy(W.qm, mf, sizeof(double) * (size_t)E * q);
            const uint8_t* z = syn ? syn + (size_t)f * M : NULL;
            one_iteration(&D, &W, z);
            sat[f] = (uint8_t)harden_and_test(&D, &W, z);
            memcpy(mf, W.qm, sizeof(double) * (size_t)E * q);
            memcpy(post + (size_t)f * N * q, W.Q, sizeof(double) * (size_t)N * q);
            for (int j = 0; j < N; j++) xhat[(size_t)f * N + j] = (uint8_t)W.xh[j];
            if (D.markov && prior_out) update_priors(&D, &W, prior_out + (size_t)f * K * q);
        }
        owork_free(&W);
    }
    oshared_free(&S);
    return err;
}

/* ----------------------------------------- entry points for unit pins */
int oracle_gf_tables(int q, unsigned poly, int32_t* mul /* [q][q] */, int32_t* inv /* [q] */) {
    ogf g;
    int rc = ogf_init(&g, q, poly);
    if (rc) return rc;
    for (int a = 0; a < q; a++)
        for (int b = 0; b < q; b++) mul[a * q + b] = gf_mul(&g, a, b);
    inv[0] = 0;
    for (int a = 1; a < q; a++) inv[a] = gf_inv(&g, a);
    return OR_OK;
}

/* Eq. 3 for one check: qin [d][q] -> rout [d][q] (normalised), by the direct
 * route (use_wht = 0) or the transform route (use_wht = 1). */
int oracle_check(int q, unsigned poly, int d, const int32_t* h, int z, const double* qin, double* rout, int use_wht) {
    ogf g;
    int rc = ogf_init(&g, q, poly);
    if (rc) return rc;
    if (d < 1 || d > 64 || z < 0 || z >= q) return OR_EINVAL;
    int hh[64];
    const double* qv[64];
    double u[256], v[256];
    for (int m = 0; m < d; m++) {
        if (h[m] <= 0 || h[m] >= q) return OR_EINVAL;
        hh[m] = h[m];
        qv[m] = qin + (size_t)m * q;
    }
    for (int k = 0; k < d; k++) {
        double* r = rout + (size_t)k * q;
        if (use_wht) check_edge_wht(&g, d, hh, qv, k, z, r, u, v);
        else check_edge_direct(&g, d, hh, qv, k, z, r, u, v);
        normalise(r, q);
    }
    return OR_OK;
}

/* Channel likelihoods of n symbols (normalised), [n][q]. */
int oracle_channel(int q, int kind, double param, int n, const float* obs, const uint8_t* punct, double* L) {
    int p = ilog2q(q);
    if (p < 0 || kind < 0 || kind > 3) return OR_EINVAL;
    int stride = kind == CH_LOGLIK ? q : p;
    for (int j = 0; j < n; j++) channel_likelihood(kind, param, q, p, obs + (size_t)j * stride, punct ? punct[j] : 0, L + (size_t)j * q);
    return OR_OK;
}

/* Markov prior of every source position from posteriors Q [K][q] (in source
 * order) by Eq. 6 (form 6) or Eq. 7 (form 7); pi_out [q] optional. */
int oracle_markov(int q, const double* T, int K, const double* Q, double* P, int form, double* pi_out) {
    if (K < 1 || q < 2 || q > 256) return OR_EINVAL;
    double* Mt = malloc(sizeof(double) * (size_t)q * q);
    double pi[256];
    if (!Mt) return OR_ENOMEM;
    for (int a = 0; a < q; a++) {
        double s = 0.0;
        for (int b = 0; b < q; b++) s += T[a * q + b];
        for (int b = 0; b < q; b++) Mt[a * q + b] = T[a * q + b] / s;
    }
    if (stationary(Mt, q, pi)) { free(Mt); return OR_EINVAL; }
    for (int i = 0; i < K; i++) {
        const double* Qm = i > 0 ? Q + (size_t)(i - 1) * q : NULL;
        const double* Qp = i < K - 1 ? Q + (size_t)(i + 1) * q : NULL;
        if (form == 7) markov_prior_eq7(Mt, pi, q, Qm, Qp, P + (size_t)i * q);
        else markov_prior_eq6(Mt, pi, q, Qm, Qp, P + (size_t)i * q);
    }
    if (pi_out) memcpy(pi_out, pi, sizeof(double) * q);
    free(Mt);
    return OR_OK;
}
