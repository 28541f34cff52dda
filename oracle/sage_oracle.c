/*
 * CPU oracle of the GPU function's hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, fp64 C loops, written from the definitions; only the tests, the
 * smoke check and the benchmark's cpu_baseline / reference arm use it.  It shares
 * no code with the CUDA path.
 *
 * The paper (SAGE, arXiv 2404.14691) does not define the GPU function itself: its
 * mechanisms (parallelised setup, Sec. 5; read-only memory sharing, Sec. 6.2)
 * produce exactly the result of running each invocation on its own.  So the
 * oracle computes, for every invocation independently, the plain definition of
 * the synthetic recommendation-style function:
 *
 *   pooled[b, t*D + d] = sum over i in bag(t,b) of W_t[idx[i], d]   (index order)
 *   h   = x;  h = ReLU(h . W_l^T + b_l)     for each bottom layer l
 *   c   = [pooled[b, 0:T*D], h]                                    (concat)
 *   g   = c;  g = ReLU(g . V_l^T + e_l)     for each top layer but the last
 *   z   = g . V_L^T + e_L;   out = 1 / (1 + exp(-z))
 *
 * Every value also carries a magnitude bound m (the same computation applied to
 * absolute values: sums of |terms|, |W| |h| + |b|); the parity checks use it as
 * the scale of the componentwise relative error (Higham, "Accuracy and Stability
 * of Numerical Algorithms", Sec. 3.1): |gpu - oracle| <= rtol * m.  For the
 * sigmoid output, m_out = s(1-s) m_z + |out| (first-order propagation plus the
 * evaluation of the sigmoid itself).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* Embedding-bag sum over one invocation (all tables, all samples).
 * tables[t]: rows x dim fp64, row-major.  offsets: [n_tables*batch + 1] table-major.
 * pooled: [batch, ldp] -- table t lands in columns [t*dim, (t+1)*dim).
 * pooled_mag (may be NULL): sum of |terms|. Returns 0, or -1 on an index out of range. */
int oracle_bag_sum(int n_tables, int batch, int dim, const double* const* tables,
                   const int64_t* table_rows, const int32_t* indices, const int64_t* offsets,
                   double* pooled, int ldp, double* pooled_mag) {
    for (int t = 0; t < n_tables; ++t) {
        for (int b = 0; b < batch; ++b) {
            int64_t g = (int64_t)t * batch + b;
            for (int d = 0; d < dim; ++d) {
                double s = 0.0, m = 0.0;
                for (int64_t i = offsets[g]; i < offsets[g + 1]; ++i) {
                    int64_t r = indices[i];
                    if (r < 0 || r >= table_rows[t]) return -1;
                    double v = tables[t][r * dim + d];
                    s += v;
                    m += fabs(v);
                }
                pooled[(int64_t)b * ldp + (int64_t)t * dim + d] = s;
                if (pooled_mag) pooled_mag[(int64_t)b * ldp + (int64_t)t * dim + d] = m;
            }
        }
    }
    return 0;
}

/* y[i, j] = act( sum_k x[i, k] * W[j, k] + bias[j] ),  W is [n, k] row-major.
 * act: 0 = identity, 1 = ReLU.  xmag/ymag (both NULL or both set) propagate the
 * magnitude bound ymag = |W| xmag + |bias|. */
void oracle_linear(int m, int k, int n, const double* x, int ldx, const double* W,
                   const double* bias, int act, double* y, int ldy,
                   const double* xmag, double* ymag) {
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < n; ++j) {
            double s = 0.0, a = 0.0;
            for (int q = 0; q < k; ++q) {
                s += x[(int64_t)i * ldx + q] * W[(int64_t)j * k + q];
                if (xmag) a += xmag[(int64_t)i * ldx + q] * fabs(W[(int64_t)j * k + q]);
            }
            s += bias[j];
            if (act == 1 && s < 0.0) s = 0.0;
            y[(int64_t)i * ldy + j] = s;
            if (ymag) ymag[(int64_t)i * ldy + j] = a + fabs(bias[j]);
        }
    }
}

double oracle_sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

/* ---- whole function, one invocation ------------------------------------- */

typedef struct {
    int n_tables, dim, n_dense;
    int n_bot, n_top;
    const int* bot_dims;           /* [n_bot] outputs */
    const int* top_dims;           /* [n_top] outputs, last == 1 */
    const double* const* bot_W;    /* [n_bot] -> [out, in] */
    const double* const* bot_b;
    const double* const* top_W;
    const double* const* top_b;
    const double* const* tables;   /* [n_tables] -> [rows, dim] */
    const int64_t* table_rows;
} oracle_fn;

typedef struct {
    const oracle_fn* fn;
    int batch;
    const double* dense;           /* [batch, n_dense] */
    const int32_t* indices;
    const int64_t* offsets;        /* [n_tables*batch+1] */
    double* out;                   /* [batch] */
    double* out_mag;               /* [batch] or NULL */
    double* pooled;                /* [batch, n_tables*dim] or NULL */
    double* pooled_mag;            /* [batch, n_tables*dim] or NULL */
    int b0, b1;                    /* sample range of this worker */
    int status;
} oracle_job;

static int max_width(const oracle_fn* f) {
    int w = f->n_dense, cd = f->n_tables * f->dim + f->bot_dims[f->n_bot - 1];
    if (cd > w) w = cd;
    for (int l = 0; l < f->n_bot; ++l) if (f->bot_dims[l] > w) w = f->bot_dims[l];
    for (int l = 0; l < f->n_top; ++l) if (f->top_dims[l] > w) w = f->top_dims[l];
    return w;
}

/* One sample b of the invocation: bottom MLP, bags, concat, top MLP, sigmoid. */
static int oracle_sample(const oracle_job* J, int b, double* h, double* hm, double* g, double* gm) {
    const oracle_fn* f = J->fn;
    int T = f->n_tables, D = f->dim, B = J->batch;
    int width = f->n_dense;
    for (int q = 0; q < f->n_dense; ++q) {
        h[q] = J->dense[(int64_t)b * f->n_dense + q];
        hm[q] = fabs(h[q]);
    }
    for (int l = 0; l < f->n_bot; ++l) {
        oracle_linear(1, width, f->bot_dims[l], h, width, f->bot_W[l], f->bot_b[l], 1, g, f->bot_dims[l], hm, gm);
        width = f->bot_dims[l];
        memcpy(h, g, sizeof(double) * width);
        memcpy(hm, gm, sizeof(double) * width);
    }
    /* concat: pooled bags of tables 0..T-1, then the bottom output */
    int cd = T * D + width;
    for (int q = 0; q < width; ++q) {
        g[T * D + q] = h[q];
        gm[T * D + q] = hm[q];
    }
    for (int t = 0; t < T; ++t) {
        int64_t bag = (int64_t)t * B + b;
        for (int d = 0; d < D; ++d) {
            double s = 0.0, m = 0.0;
            for (int64_t i = J->offsets[bag]; i < J->offsets[bag + 1]; ++i) {
                int64_t r = J->indices[i];
                if (r < 0 || r >= f->table_rows[t]) return -1;
                double v = f->tables[t][r * D + d];
                s += v;
                m += fabs(v);
            }
            g[t * D + d] = s;
            gm[t * D + d] = m;
            if (J->pooled) J->pooled[(int64_t)b * T * D + t * D + d] = s;
            if (J->pooled_mag) J->pooled_mag[(int64_t)b * T * D + t * D + d] = m;
        }
    }
    width = cd;
    for (int l = 0; l < f->n_top; ++l) {
        int last = (l == f->n_top - 1);
        oracle_linear(1, width, f->top_dims[l], g, width, f->top_W[l], f->top_b[l], last ? 0 : 1, h,
                      f->top_dims[l], gm, hm);
        width = f->top_dims[l];
        memcpy(g, h, sizeof(double) * width);
        memcpy(gm, hm, sizeof(double) * width);
    }
    double z = g[0], s = oracle_sigmoid(z);
    J->out[b] = s;
    if (J->out_mag) J->out_mag[b] = s * (1.0 - s) * gm[0] + fabs(s);
    return 0;
}

static void* oracle_worker(void* arg) {
    oracle_job* J = (oracle_job*)arg;
    int w = max_width(J->fn);
    double* buf = (double*)malloc(sizeof(double) * 4 * (size_t)w);
    J->status = 0;
    if (!buf) { J->status = -2; return NULL; }
    for (int b = J->b0; b < J->b1 && J->status == 0; ++b)
        J->status = oracle_sample(J, b, buf, buf + w, buf + 2 * w, buf + 3 * w);
    free(buf);
    return NULL;
}

/* Whole function for samples [b0, b1) of one invocation, split over n_threads
 * threads by sample (samples are independent; each is computed by the same loops).
 * Outputs are indexed by the sample's position in the invocation. */
int oracle_forward(const oracle_fn* fn, int batch, const double* dense, const int32_t* indices,
                   const int64_t* offsets, int b0, int b1, double* out, double* out_mag,
                   double* pooled, double* pooled_mag, int n_threads) {
    if (b0 < 0 || b1 > batch || b0 > b1) return -3;
    if (n_threads < 1) n_threads = 1;
    int n = b1 - b0;
    if (n_threads > n) n_threads = n > 0 ? n : 1;
    oracle_job* jobs = (oracle_job*)calloc((size_t)n_threads, sizeof(oracle_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    int rc = 0;
    for (int i = 0; i < n_threads; ++i) {
        oracle_job* J = &jobs[i];
        J->fn = fn; J->batch = batch; J->dense = dense; J->indices = indices; J->offsets = offsets;
        J->out = out; J->out_mag = out_mag; J->pooled = pooled; J->pooled_mag = pooled_mag;
        J->b0 = b0 + (int)((int64_t)n * i / n_threads);
        J->b1 = b0 + (int)((int64_t)n * (i + 1) / n_threads);
        if (n_threads == 1) oracle_worker(J);
        else pthread_create(&th[i], NULL, oracle_worker, J);
    }
    for (int i = 0; i < n_threads; ++i) {
        if (n_threads > 1) pthread_join(th[i], NULL);
        if (jobs[i].status) rc = jobs[i].status;
    }
    free(jobs);
    free(th);
    return rc;
}
