/*
 * Oracle: plain FP64 CPU evaluation of the UDF predicates.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA path is
 * compared with; it shares no code, header or constant with the CUDA path,
 * and the product never links, loads or calls it.
 *
 * What it computes is the plain definition of a conjunction of UDF
 * predicates (Sec. 1, Listing 1; Sec. 3.2): every UDF is evaluated on every
 * tuple, in FP64, by direct loops.  The method under test reaches the same
 * pass set faster by ordering and short-circuiting (Sec. 3.3 "Eager
 * Materialization"); the oracle does neither.
 *
 *  - MLP UDF:  h_{l+1} = W_l h_l + b_l, ReLU on every layer but the last; the
 *    last layer has one output, the score.
 *  - CNN UDF:  input x/255 (uint8 CHW frame), conv 3x3 stride 1 zero-pad 1
 *    + bias + ReLU per layer, global average pool over H*W, then
 *    score = head_w . pooled + head_b.
 *
 * Weights arrive as fp32 (the generated values); they are widened to FP64
 * exactly.  Summation runs in FP64 in loop order; the order is not part of
 * the definition and only moves the last bits.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------ threading */

typedef struct {
    int64_t n;
    int64_t next;             /* next item, claimed under the lock */
    pthread_mutex_t lock;
    void (*item)(void *ctx, int64_t i, double *scratch);
    void *ctx;
    size_t scratch_doubles;
    int failed;
} pool_t;

static void *worker(void *arg) {
    pool_t *p = (pool_t *)arg;
    double *scratch = (double *)malloc(p->scratch_doubles * sizeof(double) + 64);
    if (!scratch) {
        pthread_mutex_lock(&p->lock);
        p->failed = 1;
        pthread_mutex_unlock(&p->lock);
        return NULL;
    }
    for (;;) {
        pthread_mutex_lock(&p->lock);
        int64_t i = p->next++;
        pthread_mutex_unlock(&p->lock);
        if (i >= p->n) break;
        p->item(p->ctx, i, scratch);
    }
    free(scratch);
    return NULL;
}

static int run_items(int64_t n, int n_threads, size_t scratch_doubles,
                     void (*item)(void *, int64_t, double *), void *ctx) {
    if (n_threads <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        n_threads = c > 0 ? (int)c : 1;
    }
    if (n_threads > n) n_threads = (int)(n > 0 ? n : 1);
    pool_t p;
    p.n = n;
    p.next = 0;
    pthread_mutex_init(&p.lock, NULL);
    p.item = item;
    p.ctx = ctx;
    p.scratch_doubles = scratch_doubles;
    p.failed = 0;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    if (!th) return -1;
    int started = 0;
    for (int t = 0; t < n_threads; ++t) {
        if (pthread_create(&th[t], NULL, worker, &p) != 0) break;
        ++started;
    }
    if (started == 0) worker(&p);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&p.lock);
    return p.failed ? -1 : 0;
}

int oracle_threads(void) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/* ------------------------------------------------------------------ MLP */

typedef struct {
    const float *X;
    int64_t ld;
    int n_layers;
    const int32_t *dims;
    const float *const *W;
    const float *const *b;
    double *out;
    int width_max;
} mlp_ctx;

static void mlp_item(void *vc, int64_t t, double *scratch) {
    const mlp_ctx *c = (const mlp_ctx *)vc;
    double *h = scratch;                       /* current activations */
    double *g = scratch + c->width_max;        /* next activations */
    const float *x = c->X + t * c->ld;
    for (int k = 0; k < c->dims[0]; ++k) h[k] = (double)x[k];
    for (int l = 0; l < c->n_layers; ++l) {
        const int fi = c->dims[l], fo = c->dims[l + 1];
        const float *W = c->W[l];
        const float *b = c->b[l];
        for (int j = 0; j < fo; ++j) {
            double s = (double)b[j];
            const float *w = W + (int64_t)j * fi;
            for (int k = 0; k < fi; ++k) s += (double)w[k] * h[k];
            /* ReLU on hidden layers only; the last layer is the score */
            g[j] = (l + 1 < c->n_layers && s < 0.0) ? 0.0 : s;
        }
        double *tmp = h; h = g; g = tmp;
    }
    c->out[t] = h[0];
}

/* Scores of one MLP UDF on n rows of X (row stride ld floats).
 * dims has n_layers+1 entries and dims[n_layers] must be 1.
 * W[l] is [dims[l+1] x dims[l]] row-major, b[l] is [dims[l+1]].
 * Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_mlp_scores(const float *X, int64_t n, int64_t ld, int n_layers,
                      const int32_t *dims, const float *const *W,
                      const float *const *b, double *out, int n_threads) {
    if (!X || !dims || !W || !b || !out || n < 0 || n_layers < 1) return -1;
    if (dims[n_layers] != 1 || ld < dims[0]) return -1;
    int wmax = 1;
    for (int l = 0; l <= n_layers; ++l) {
        if (dims[l] < 1) return -1;
        if (dims[l] > wmax) wmax = dims[l];
    }
    mlp_ctx c = {X, ld, n_layers, dims, W, b, out, wmax};
    return run_items(n, n_threads, (size_t)2 * wmax, mlp_item, &c);
}

/* ------------------------------------------------------------------ CNN */

typedef struct {
    const uint8_t *frames;
    int C0, H, W;
    int n_conv;
    const int32_t *ch;
    const float *const *Wc;
    const float *const *bc;
    const float *hw;
    double hb;
    double *out;
    int cmax;
} cnn_ctx;

/* One frame: activations kept as zero-padded planes [C][(H+2) x (W+2)] so
 * that the 3x3 taps at the border read the padding zeros. */
static void cnn_item(void *vc, int64_t t, double *scratch) {
    const cnn_ctx *c = (const cnn_ctx *)vc;
    const int H = c->H, W = c->W, HP = H + 2, WP = W + 2;
    const size_t plane = (size_t)HP * WP;
    double *a = scratch;                              /* input, padded  */
    double *o = scratch + (size_t)c->cmax * plane;    /* output, padded */
    memset(a, 0, sizeof(double) * (size_t)c->cmax * plane);
    memset(o, 0, sizeof(double) * (size_t)c->cmax * plane);

    const uint8_t *f = c->frames + (size_t)t * c->C0 * H * W;
    for (int ci = 0; ci < c->C0; ++ci)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                a[ci * plane + (size_t)(y + 1) * WP + (x + 1)] =
                    (double)f[((size_t)ci * H + y) * W + x] / 255.0;

    for (int l = 0; l < c->n_conv; ++l) {
        const int Ci = c->ch[l], Co = c->ch[l + 1];
        const float *Wl = c->Wc[l];
        const float *bl = c->bc[l];
        for (int co = 0; co < Co; ++co) {
            double *op = o + co * plane;
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x)
                    op[(size_t)(y + 1) * WP + (x + 1)] = (double)bl[co];
            for (int ci = 0; ci < Ci; ++ci) {
                const double *ip = a + ci * plane;
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx) {
                        /* weight W[co][ci][ky][kx] multiplies in[y+ky-1][x+kx-1] */
                        const double w = (double)Wl[(((size_t)co * Ci + ci) * 3 + ky) * 3 + kx];
                        for (int y = 0; y < H; ++y) {
                            double *orow = op + (size_t)(y + 1) * WP + 1;
                            const double *irow = ip + (size_t)(y + ky) * WP + kx;
                            for (int x = 0; x < W; ++x) orow[x] += w * irow[x];
                        }
                    }
            }
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    double *v = &op[(size_t)(y + 1) * WP + (x + 1)];
                    if (*v < 0.0) *v = 0.0;                       /* ReLU */
                }
        }
        double *tmp = a; a = o; o = tmp;
    }

    const int CL = c->ch[c->n_conv];
    double s = c->hb;
    for (int ch = 0; ch < CL; ++ch) {
        double sum = 0.0;
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) sum += a[ch * plane + (size_t)(y + 1) * WP + (x + 1)];
        s += (double)c->hw[ch] * (sum / (double)(H * W));          /* global average pool */
    }
    c->out[t] = s;
}

/* Scores of one CNN UDF on n uint8 frames [n][C0][H][W].
 * ch has n_conv+1 entries (ch[0] == C0); Wc[l] is [ch[l+1]][ch[l]][3][3],
 * bc[l] is [ch[l+1]]; hw is [ch[n_conv]].  Returns 0 or -1. */
int oracle_cnn_scores(const uint8_t *frames, int64_t n, int C0, int H, int W,
                      int n_conv, const int32_t *ch, const float *const *Wc,
                      const float *const *bc, const float *hw, double hb,
                      double *out, int n_threads) {
    if (!frames || !ch || !Wc || !bc || !hw || !out || n < 0 || n_conv < 1) return -1;
    if (H < 1 || W < 1 || ch[0] != C0) return -1;
    int cmax = 1;
    for (int l = 0; l <= n_conv; ++l) {
        if (ch[l] < 1) return -1;
        if (ch[l] > cmax) cmax = ch[l];
    }
    cnn_ctx c = {frames, C0, H, W, n_conv, ch, Wc, bc, hw, hb, out, cmax};
    return run_items(n, n_threads, (size_t)2 * cmax * (H + 2) * (W + 2), cnn_item, &c);
}
