/*
 * Seeded, counter-based input generator shared by the CUDA path and the CPU oracle.
 *
 * It produces the read-only data of a synthetic recommendation-style GPU function:
 * embedding tables and MLP weights.  It holds none of the method's arithmetic; it
 * only defines what the inputs are, so that both sides can read exactly the same
 * values without either one producing them for the other.
 *
 * Random source: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a counter-based generator:
 * draw(seed, e) is the (e+1)-th output of the SplitMix64 sequence started at `seed`,
 * i.e. mix64(seed + (e+1) * 0x9E3779B97F4A7C15).
 *
 * Value of element e of a stream with half-width `bound` (uniform on [-bound, bound)):
 *     k = (draw(seed, e) >> 40) - 2^23            (a signed 24-bit integer)
 *     v = (float)k * step,  step = (float)bound / 2^23   (one fp32 rounding)
 * BF16 data stores v rounded to nearest-even to bfloat16.
 *
 * Blob layouts (they match the layouts the C-ABI documents for sage_fn_desc):
 *   tables blob : table t (rows[t] x dim elements, row-major) follows table t-1
 *                 with no padding.
 *   weights blob: for each layer l (bottom layers, then top layers):
 *                 W_l [out_l x in_l] in the table dtype, then b_l [out_l] fp32;
 *                 each of the two arrays starts at a 256-byte aligned offset.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>

#define WL_GAMMA 0x9E3779B97F4A7C15ULL

/* The loops below call these internal copies: the exported symbols can be
 * interposed in a shared library, which would keep the compiler from inlining
 * (and vectorising) them.  Same arithmetic, same values. */
static inline uint64_t mix64_(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t wl_mix64(uint64_t z) { return mix64_(z); }

uint64_t wl_draw(uint64_t seed, uint64_t e) { return mix64_(seed + (e + 1) * WL_GAMMA); }


static inline uint16_t wl_bf16_rne(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

/* Fill n elements [first, first+n) of stream (seed, bound); dtype 0 = fp32, 1 = bf16. */
__attribute__((target_clones("arch=x86-64-v4", "arch=x86-64-v3", "default")))
void wl_fill_stream(void* dst, int dtype, uint64_t seed, float bound, uint64_t first, size_t n) {
    float step = bound / 8388608.0f;
    /* the SplitMix64 state of element e is seed + (e + 1) * gamma: advanced by one
     * addition per element (the same values as computing it from e each time) */
    uint64_t z = seed + (first + 1) * WL_GAMMA;
    if (dtype == 0) {
        float* d = (float*)dst;
        for (size_t i = 0; i < n; ++i, z += WL_GAMMA) d[i] = (float)((int32_t)(mix64_(z) >> 40) - 8388608) * step;
    } else {
        uint16_t* d = (uint16_t*)dst;
        for (size_t i = 0; i < n; ++i, z += WL_GAMMA)
            d[i] = wl_bf16_rne((float)((int32_t)(mix64_(z) >> 40) - 8388608) * step);
    }
}

/* ---- tables blob -------------------------------------------------------- */

typedef struct {
    int n_tables;
    int dim;
    int dtype;               /* 0 fp32, 1 bf16 */
    float bound;             /* half-width of the uniform distribution */
    const int64_t* rows;     /* [n_tables] */
    const uint64_t* seeds;   /* [n_tables] */
    int fail_at_call;        /* test hook: return -1 on this call number (0 = never) */
    int calls;               /* counts calls when fail_at_call != 0 */
} wl_tables_ctx;

/* Fill bytes [off, off+n) of the tables blob.  off and n must be multiples of the
 * element size.  Returns 0 on success, -1 on a bad range. Signature matches the
 * C-ABI's producer callback. */
int wl_fill_tables(void* dst, size_t off, size_t n, void* vctx) {
    wl_tables_ctx* c = (wl_tables_ctx*)vctx;
    size_t es = c->dtype == 0 ? 4 : 2;
    if (c->fail_at_call) {
        int call = __atomic_add_fetch(&c->calls, 1, __ATOMIC_SEQ_CST);
        if (call >= c->fail_at_call) return -1;
    }
    if (off % es || n % es) return -1;
    uint64_t e0 = off / es, ne = n / es;
    char* out = (char*)dst;
    uint64_t tbeg = 0;
    for (int t = 0; t < c->n_tables && ne > 0; ++t) {
        uint64_t tn = (uint64_t)c->rows[t] * (uint64_t)c->dim;
        uint64_t tend = tbeg + tn;
        if (e0 < tend) {
            uint64_t first = e0 - tbeg;
            uint64_t take = tend - e0;
            if (take > ne) take = ne;
            wl_fill_stream(out, c->dtype, c->seeds[t], c->bound, first, (size_t)take);
            out += take * es;
            e0 += take;
            ne -= take;
        }
        tbeg = tend;
    }
    return ne == 0 ? 0 : -1;
}

/* ---- weights blob -------------------------------------------------------- */

typedef struct {
    int n_layers;
    int dtype;                 /* dtype of W; biases are always fp32 */
    const int* in_dims;        /* [n_layers] */
    const int* out_dims;       /* [n_layers] */
    const uint64_t* w_seeds;   /* [n_layers] */
    const uint64_t* b_seeds;   /* [n_layers] */
} wl_weights_ctx;

static size_t wl_align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t wl_weights_bytes(const wl_weights_ctx* c) {
    size_t es = c->dtype == 0 ? 4 : 2, o = 0;
    for (int l = 0; l < c->n_layers; ++l) {
        o = wl_align256(o) + (size_t)c->out_dims[l] * c->in_dims[l] * es;
        o = wl_align256(o) + (size_t)c->out_dims[l] * 4;
    }
    return wl_align256(o);
}

/* Fill the whole weights blob into dst (zeroing the padding).  Xavier-uniform
 * weights, bound sqrt(6/(in+out)); biases uniform with bound 1/sqrt(in). */
int wl_fill_weights_full(void* dst, void* vctx) {
    wl_weights_ctx* c = (wl_weights_ctx*)vctx;
    size_t es = c->dtype == 0 ? 4 : 2, o = 0;
    memset(dst, 0, wl_weights_bytes(c));
    for (int l = 0; l < c->n_layers; ++l) {
        size_t nw = (size_t)c->out_dims[l] * c->in_dims[l];
        float wb = (float)sqrt(6.0 / (double)(c->in_dims[l] + c->out_dims[l]));
        float bb = (float)(1.0 / sqrt((double)c->in_dims[l]));
        o = wl_align256(o);
        wl_fill_stream((char*)dst + o, c->dtype, c->w_seeds[l], wb, 0, nw);
        o += nw * es;
        o = wl_align256(o);
        wl_fill_stream((char*)dst + o, 0, c->b_seeds[l], bb, 0, (size_t)c->out_dims[l]);
        o += (size_t)c->out_dims[l] * 4;
    }
    return 0;
}

/* Fill `n` rows (rows[i] of one table stream) of `dim` elements each into dst,
 * row after row; used by the oracle to read only the rows a check needs. */
void wl_fill_rows(void* dst, int dtype, uint64_t seed, float bound, int dim,
                  const int64_t* rows, size_t n) {
    size_t es = dtype == 0 ? 4 : 2;
    for (size_t i = 0; i < n; ++i)
        wl_fill_stream((char*)dst + i * (size_t)dim * es, dtype, seed, bound,
                       (uint64_t)rows[i] * (uint64_t)dim, (size_t)dim);
}
