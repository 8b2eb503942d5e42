/*
 * szx_ref.c -- CPU oracle of the SZx block codec (arXiv 2201.13020).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE: only tests/, __graft_entry__.smoke()
 * and bench.py's cpu_baseline / reference arm may build, load or run it.  It
 * shares nothing with the CUDA path.  It is deliberately plain and slow: one
 * value at a time, one block at a time, in the paper's order.
 *
 * ---------------------------------------------------------------------------
 * What the paper fixes (Sec. III-IV, Algorithm 1, Eq. 4, Eq. 5):
 *   - the data are cut into consecutive 1-D blocks of b values (Alg. 1, loop
 *     over blocks; b = 128 by default, Sec. V-A.2);
 *   - mu_k is the mean of the block's min and max, r_k its variation radius
 *     (Table 1);
 *   - a block is "constant" iff every |d_i - mu_k| <= e; it then stores only
 *     mu_k (Alg. 1, constant branch);
 *   - otherwise values are normalised, v_i = d_i - mu_k, and keep the bits
 *     that Eq. 4 requires; Eq. 5 right-shifts them so the kept bits fill
 *     whole bytes (Sec. V-A, "Solution C");
 *   - v_i is XORed with v_{i-1}; the number of identical leading bytes
 *     (0..3) is a 2-bit code in the lead-code array, and only the remaining
 *     "mid-bytes" go to the mid-byte array (the bullets after Alg. 1);
 *   - |d_i - d'_i| <= e for every value (Eq. 1).
 *
 * Readings where the paper is silent, garbled or loose (each one is listed
 * in the design notes of the repository):
 *   R1  mu = RN(mn + r) with r = RN(RN(mx - mn) * 0.5), in the value's own
 *       precision.  The sentence after Alg. 1 says "subtracting the variation
 *       radius (i.e. mean of min and max)"; it means subtracting mu.
 *   R2  min/max use IEEE totalOrder on finite values (-0 < +0), so they do not
 *       depend on the scan order.  A block holding a NaN or an infinity, or
 *       whose r or mu overflows, is stored raw (verbatim).
 *   R3  The constant test of Alg. 1 is evaluated exactly (no rounding of
 *       d_i - mu) with an error-free transform.
 *   R4  e for f32 is the largest float <= eb (rounded toward zero); for f64
 *       e = eb.  p(x) in Eq. 4 is the unbiased exponent field of x (zero and
 *       subnormals give the field's minimum, 0 - bias).
 *   R5  Eq. 4's clamp "sizeof(type)" is the mantissa width M (23 / 52): R_k
 *       counts mantissa bits, and sign + exponent (1 + E bits) are always
 *       kept, so reqBits = 1 + E + R_k.
 *   R6  Eq. 5 is applied to reqBits (not to R_k alone): s = (8 - reqBits % 8)
 *       % 8, so that the kept prefix is q = (reqBits + s) / 8 whole bytes.
 *       t_i = (bits(v_i) >> s) masked to its top 8q bits; the decoder uses
 *       v'_i = t_i << s and d'_i = RN(v'_i + mu).
 *   R7  The paper claims strict error control but gives no rounding analysis;
 *       RN in v = d - mu and in d' = v' + mu can push |d - d'| past e.  So a
 *       block is checked value by value (exactly); if one value fails,
 *       reqBits grows by one and the block is re-encoded; a block that still
 *       fails at full width is stored raw.
 *   R8  XOR is taken between the truncated words t_i and t_{i-1} (the only
 *       thing a decoder has), with t_{-1} = 0 in every block, and the
 *       identical-leading-byte count is L_i = min(clz_bytes(t_i ^ t_{i-1}),
 *       3, q).
 *   R9  Layout (ours; the paper fixes none): a value's mid-bytes are bytes
 *       L_i .. q-1 of t_i (byte 0 = most significant).  Inside a block they
 *       are written plane by plane: plane j holds byte j of every t_i with
 *       L_i <= j, in ascending i, planes j = 0 .. q-1 in order.  Same byte
 *       count as the paper's value-major mb_array.
 *   R10 Stream = 64-byte header | state bitmap | mu array | tile index |
 *       tile records, each section zero-padded to 16 bytes (all little
 *       endian).  A tile is G = max(8, 32768 / (b * w)) consecutive blocks.
 *       Tile record = lead codes of its non-constant blocks (b/4 bytes each)
 *       | their reqBits bytes (0xFF = raw) | their mid-bytes (a raw block
 *       contributes its len * w input bytes) | zero pad to 16.  The tile
 *       index holds each record's offset from the first record, plus the
 *       total, so tiles decode independently.
 *   R11 A partial last block is coded with its true length; its unused
 *       lead codes are 0.
 * ---------------------------------------------------------------------------
 */
#include "szx_ref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- floating-point formats -------------------------------------------- */

typedef struct {
    int w;    /* bytes per value */
    int W;    /* bits per value */
    int E;    /* exponent bits */
    int M;    /* mantissa bits */
    int bias; /* exponent bias */
} fmt_t;

static const fmt_t FMT_F32 = {4, 32, 8, 23, 127};
static const fmt_t FMT_F64 = {8, 64, 11, 52, 1023};

static const fmt_t *fmt_of(int dtype)
{
    if (dtype == SZX_REF_F32) return &FMT_F32;
    if (dtype == SZX_REF_F64) return &FMT_F64;
    return NULL;
}

/* Values are handled as their bit patterns held in a uint64_t. */

static float as_f32(uint64_t u) { uint32_t x = (uint32_t)u; float f; memcpy(&f, &x, 4); return f; }
static uint64_t of_f32(float f) { uint32_t x; memcpy(&x, &f, 4); return x; }
static double as_f64(uint64_t u) { double d; memcpy(&d, &u, 8); return d; }
static uint64_t of_f64(double d) { uint64_t x; memcpy(&x, &d, 8); return x; }

static uint64_t load_value(const fmt_t *f, const uint8_t *p)
{
    uint64_t x = 0;
    for (int i = 0; i < f->w; i++) x |= (uint64_t)p[i] << (8 * i);
    return x;
}

static void store_value(const fmt_t *f, uint8_t *p, uint64_t x)
{
    for (int i = 0; i < f->w; i++) p[i] = (uint8_t)(x >> (8 * i));
}

static int is_finite(const fmt_t *f, uint64_t a)
{
    uint64_t expo = (a >> f->M) & ((1u << f->E) - 1);
    return expo != (uint64_t)((1u << f->E) - 1);
}

static int sign_bit(const fmt_t *f, uint64_t a) { return (int)((a >> (f->W - 1)) & 1); }

/* p(x) of Eq. 4: the exponent field minus the bias (reading R4). */
static int exponent_of(const fmt_t *f, uint64_t a)
{
    return (int)((a >> f->M) & ((1u << f->E) - 1)) - f->bias;
}

/* Round-to-nearest-even arithmetic in the value's own precision. */
static uint64_t sub_rn(const fmt_t *f, uint64_t a, uint64_t b)
{
    if (f->w == 4) return of_f32(as_f32(a) - as_f32(b));
    return of_f64(as_f64(a) - as_f64(b));
}

static uint64_t add_rn(const fmt_t *f, uint64_t a, uint64_t b)
{
    if (f->w == 4) return of_f32(as_f32(a) + as_f32(b));
    return of_f64(as_f64(a) + as_f64(b));
}

static uint64_t half_rn(const fmt_t *f, uint64_t a)
{
    if (f->w == 4) return of_f32(as_f32(a) * 0.5f);
    return of_f64(as_f64(a) * 0.5);
}

/* totalOrder on finite values: numeric order, and -0 before +0 (R2). */
static int total_less(const fmt_t *f, uint64_t a, uint64_t b)
{
    double x = (f->w == 4) ? (double)as_f32(a) : as_f64(a);
    double y = (f->w == 4) ? (double)as_f32(b) : as_f64(b);
    if (x < y) return 1;
    if (x > y) return 0;
    return sign_bit(f, a) && !sign_bit(f, b);
}

/*
 * Exact test |a - b| <= e for finite a, b and finite e >= 0 (R3, R7).
 * s = RN(a - b).  If |s| < e the exact difference is <= e (RN is monotone and
 * e is representable); if |s| > e it is > e.  Only when |s| == e does the
 * rounding error matter; it is recovered exactly by Knuth's TwoSum, and the
 * difference is <= e iff that error does not point away from zero.  The test
 * never answers "yes" wrongly; an overflow inside TwoSum (only possible for
 * operands near the format's maximum) makes it answer "no".
 */
static int within_exact(const fmt_t *f, uint64_t a, uint64_t b, uint64_t e)
{
    if (f->w == 4) {
        float x = as_f32(a), y = -as_f32(b), eb = as_f32(e);
        float s = x + y;
        if (isinf(s)) return 0;
        if (fabsf(s) < eb) return 1;
        if (fabsf(s) > eb) return 0;
        float bv = s - x;
        float av = s - bv;
        float t = (x - av) + (y - bv);
        if (s > 0) return t <= 0.0f;
        if (s < 0) return t >= 0.0f;
        return t == 0.0f;
    } else {
        double x = as_f64(a), y = -as_f64(b), eb = as_f64(e);
        double s = x + y;
        if (isinf(s)) return 0;
        if (fabs(s) < eb) return 1;
        if (fabs(s) > eb) return 0;
        double bv = s - x;
        double av = s - bv;
        double t = (x - av) + (y - bv);
        if (s > 0) return t <= 0.0;
        if (s < 0) return t >= 0.0;
        return t == 0.0;
    }
}

/* The f32 bound is the largest float <= eb (R4). */
uint64_t szx_ref_error_bound_bits(double eb, int dtype)
{
    if (dtype == SZX_REF_F64) return of_f64(eb);
    float e = (float)eb;
    if ((double)e > eb) e = nextafterf(e, 0.0f);
    return of_f32(e);
}

/* ---- stream geometry ---------------------------------------------------- */

static size_t pad16(size_t x) { return (x + 15) & ~(size_t)15; }

static int block_ok(uint32_t b)
{
    return b >= 32 && b <= 1024 && (b & (b - 1)) == 0;
}

static size_t tile_blocks_of(const fmt_t *f, uint32_t b)
{
    size_t g = 32768 / ((size_t)b * (size_t)f->w);
    return g < 8 ? 8 : g;
}

typedef struct {
    size_t n, nb, G, ntiles;
    size_t off_state, off_mu, off_index, off_rec;
} geom_t;

static void geometry(const fmt_t *f, size_t n, uint32_t b, size_t G, geom_t *g)
{
    g->n = n;
    g->nb = (n + b - 1) / b;
    g->G = G;
    g->ntiles = (g->nb + G - 1) / G;
    g->off_state = 64;
    g->off_mu = g->off_state + pad16((g->nb + 7) / 8);
    g->off_index = g->off_mu + pad16(g->nb * (size_t)f->w);
    g->off_rec = g->off_index + pad16((g->ntiles + 1) * 8);
}

size_t szx_ref_compress_bound(size_t n, int dtype, uint32_t block)
{
    const fmt_t *f = fmt_of(dtype);
    if (!f || !block_ok(block) || n == 0) return 0;
    geom_t g;
    geometry(f, n, block, tile_blocks_of(f, block), &g);
    /* worst case: every block raw */
    size_t total = g.off_rec;
    for (size_t t = 0; t < g.ntiles; t++) {
        size_t k0 = t * g.G, k1 = k0 + g.G < g.nb ? k0 + g.G : g.nb;
        size_t v0 = k0 * block, v1 = k1 * block < n ? k1 * block : n;
        total += pad16((k1 - k0) * (block / 4 + 1) + (v1 - v0) * (size_t)f->w);
    }
    return total;
}

/* ---- one block (Algorithm 1, loop body) --------------------------------- */

enum { KIND_CONST = 0, KIND_NONCONST = 1, KIND_RAW = 2 };

typedef struct {
    int kind;
    uint64_t mu;      /* mu bits (0 for raw blocks) */
    int req;          /* reqBits, or 0xFF for raw */
    int escalated;    /* reqBits grew past 1 + E + R_k */
    size_t mid_len;   /* mid bytes written */
} block_out_t;

static uint64_t top_mask(const fmt_t *f, int q)
{
    int keep = 8 * q;
    if (keep >= f->W) return f->W == 64 ? ~(uint64_t)0 : 0xFFFFFFFFull;
    uint64_t all = f->W == 64 ? ~(uint64_t)0 : 0xFFFFFFFFull;
    return (all << (f->W - keep)) & all;
}

/* number of identical leading bytes of x and y, i.e. zero leading bytes of x ^ y */
static int lead_zero_bytes(const fmt_t *f, uint64_t x)
{
    int nz = 0;
    for (int j = 0; j < f->w; j++) {
        uint8_t byte = (uint8_t)(x >> (f->W - 8 - 8 * j));
        if (byte != 0) break;
        nz++;
    }
    return nz;
}

static uint8_t byte_j(const fmt_t *f, uint64_t t, int j)
{
    return (uint8_t)(t >> (f->W - 8 - 8 * j));
}

/*
 * Encode one block of len values.  lead receives b/4 bytes, mid receives the
 * block's mid bytes (capacity len * w).  work holds 2 * len uint64 scratch.
 */
static void encode_block(const fmt_t *f, const uint8_t *vals, size_t len,
                         uint32_t b, uint64_t e, uint8_t *lead, uint8_t *mid,
                         uint64_t *work, block_out_t *o)
{
    uint64_t *v = work;        /* normalised values v_i */
    uint64_t *t = work + len;  /* truncated, shifted words t_i */
    memset(lead, 0, b / 4);
    o->escalated = 0;
    o->mid_len = 0;

    int finite = 1;
    for (size_t i = 0; i < len; i++)
        if (!is_finite(f, load_value(f, vals + i * f->w))) finite = 0;

    uint64_t mn = 0, mx = 0, r = 0, mu = 0;
    if (finite) {
        /* Alg. 1: compute mu_k, the mean of min and max (R1, R2) */
        mn = mx = load_value(f, vals);
        for (size_t i = 1; i < len; i++) {
            uint64_t x = load_value(f, vals + i * f->w);
            if (total_less(f, x, mn)) mn = x;
            if (total_less(f, mx, x)) mx = x;
        }
        r = half_rn(f, sub_rn(f, mx, mn));
        mu = add_rn(f, mn, r);
        if (!is_finite(f, r) || !is_finite(f, mu)) finite = 0;
    }
    if (!finite) goto raw;

    /* Alg. 1: constant block iff every |d_i - mu_k| <= e (R3) */
    {
        int constant = 1;
        for (size_t i = 0; i < len && constant; i++)
            if (!within_exact(f, load_value(f, vals + i * f->w), mu, e)) constant = 0;
        if (constant) {
            o->kind = KIND_CONST;
            o->mu = mu;
            o->req = 0;
            return;
        }
    }

    /* Eq. 4: required mantissa bits R_k, clamped to [0, M] (R4, R5) */
    int R = exponent_of(f, r) - exponent_of(f, e);
    if (R < 0) R = 0;
    if (R > f->M) R = f->M;
    int req0 = 1 + f->E + R;

    /* normalisation by mu */
    for (size_t i = 0; i < len; i++)
        v[i] = sub_rn(f, load_value(f, vals + i * f->w), mu);

    /* Eq. 5 right shift, truncation, and the per-value check (R6, R7) */
    int req = req0, ok = 0, q = 0, s = 0;
    for (; req <= f->W; req++) {
        s = (8 - req % 8) % 8;
        q = (req + s) / 8;
        uint64_t mask = top_mask(f, q);
        ok = 1;
        for (size_t i = 0; i < len; i++) {
            t[i] = (v[i] >> s) & mask;
            uint64_t vp = t[i] << s;
            if (f->W == 32) vp &= 0xFFFFFFFFull;
            uint64_t dp = add_rn(f, vp, mu);
            if (!within_exact(f, load_value(f, vals + i * f->w), dp, e)) ok = 0;
        }
        if (ok) break;
    }
    if (!ok) goto raw;

    o->kind = KIND_NONCONST;
    o->mu = mu;
    o->req = req;
    o->escalated = req > req0;

    /* identical leading bytes against the previous truncated word (R8) */
    {
        int lmax = q < 3 ? q : 3;
        uint64_t prev = 0;
        uint8_t *L = (uint8_t *)v; /* v no longer needed: reuse as L_i storage */
        for (size_t i = 0; i < len; i++) {
            int l = lead_zero_bytes(f, t[i] ^ prev);
            if (l > lmax) l = lmax;
            L[i] = (uint8_t)l;
            lead[i >> 2] |= (uint8_t)(l << (2 * (i & 3)));
            prev = t[i];
        }
        /* mid-bytes, plane by plane (R9) */
        for (int j = 0; j < q; j++)
            for (size_t i = 0; i < len; i++)
                if (L[i] <= j) mid[o->mid_len++] = byte_j(f, t[i], j);
    }
    return;

raw:
    o->kind = KIND_RAW;
    o->mu = 0;
    o->req = 0xFF;
    memcpy(mid, vals, len * f->w);
    o->mid_len = len * f->w;
}

/* ---- whole stream -------------------------------------------------------- */

static void put_u32(uint8_t *p, uint32_t x) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(x >> (8 * i)); }
static void put_u64(uint8_t *p, uint64_t x) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(x >> (8 * i)); }
static uint32_t get_u32(const uint8_t *p) { uint32_t x = 0; for (int i = 0; i < 4; i++) x |= (uint32_t)p[i] << (8 * i); return x; }
static uint64_t get_u64(const uint8_t *p) { uint64_t x = 0; for (int i = 0; i < 8; i++) x |= (uint64_t)p[i] << (8 * i); return x; }

#define SZX_MAGIC 0x42585A53u /* "SZXB" */
#define SZX_VERSION 1

int szx_ref_compress(const void *in, size_t n, int dtype, double eb,
                     uint32_t block, void *out, size_t cap, size_t *out_bytes)
{
    const fmt_t *f = fmt_of(dtype);
    if (!f || !in || !out || !out_bytes || n == 0 || !block_ok(block)) return SZX_REF_ERR_INVALID;
    if (!(eb > 0.0) || isinf(eb) || isnan(eb)) return SZX_REF_ERR_INVALID;
    size_t bound = szx_ref_compress_bound(n, dtype, block);
    if (cap < bound) return SZX_REF_ERR_TOO_SMALL;

    const uint8_t *src = (const uint8_t *)in;
    uint8_t *dst = (uint8_t *)out;
    uint64_t e = szx_ref_error_bound_bits(eb, dtype);
    geom_t g;
    geometry(f, n, block, tile_blocks_of(f, block), &g);
    memset(dst, 0, g.off_rec);

    uint8_t *lead = (uint8_t *)malloc(g.G * (block / 4));
    uint8_t *reqs = (uint8_t *)malloc(g.G);
    uint8_t *mids = (uint8_t *)malloc(g.G * block * (size_t)f->w);
    uint64_t *work = (uint64_t *)malloc(2 * block * sizeof(uint64_t));
    if (!lead || !reqs || !mids || !work) {
        free(lead); free(reqs); free(mids); free(work);
        return SZX_REF_ERR_INVALID;
    }

    uint64_t nn = 0, nraw = 0, nesc = 0;
    size_t rec = 0; /* running offset of the next tile record */
    for (size_t tile = 0; tile < g.ntiles; tile++) {
        size_t k0 = tile * g.G;
        size_t k1 = k0 + g.G < g.nb ? k0 + g.G : g.nb;
        size_t nn_t = 0, mid_t = 0;
        put_u64(dst + g.off_index + 8 * tile, rec);
        for (size_t k = k0; k < k1; k++) {
            size_t first = k * block;
            size_t len = first + block <= n ? block : n - first;
            block_out_t o;
            encode_block(f, src + first * f->w, len, block, e,
                         lead + nn_t * (block / 4), mids + mid_t, work, &o);
            store_value(f, dst + g.off_mu + k * f->w, o.mu);
            if (o.kind == KIND_CONST) continue;
            dst[g.off_state + k / 8] |= (uint8_t)(1u << (k % 8));
            reqs[nn_t] = (uint8_t)o.req;
            mid_t += o.mid_len;
            nn_t++;
            nn++;
            if (o.kind == KIND_RAW) nraw++;
            if (o.escalated) nesc++;
        }
        /* tile record: lead codes | reqBits bytes | mid bytes | zero pad (R10) */
        uint8_t *p = dst + g.off_rec + rec;
        size_t lead_bytes = nn_t * (block / 4);
        memcpy(p, lead, lead_bytes);
        memcpy(p + lead_bytes, reqs, nn_t);
        memcpy(p + lead_bytes + nn_t, mids, mid_t);
        size_t used = lead_bytes + nn_t + mid_t;
        memset(p + used, 0, pad16(used) - used);
        rec += pad16(used);
    }
    put_u64(dst + g.off_index + 8 * g.ntiles, rec);
    free(lead); free(reqs); free(mids); free(work);

    size_t total = g.off_rec + rec;
    memset(dst, 0, 64);
    put_u32(dst + 0, SZX_MAGIC);
    dst[4] = SZX_VERSION;
    dst[5] = (uint8_t)dtype;
    put_u32(dst + 8, block);
    put_u32(dst + 12, (uint32_t)g.G);
    put_u64(dst + 16, n);
    put_u64(dst + 24, e);
    put_u64(dst + 32, nn);
    put_u64(dst + 40, nraw);
    put_u64(dst + 48, nesc);
    put_u64(dst + 56, total);
    *out_bytes = total;
    return SZX_REF_OK;
}

/* ---- decompression (the exact inverse) ----------------------------------- */

int szx_ref_decompress(const void *in, size_t in_bytes, void *out, size_t cap,
                       size_t *n_out, int *dtype_out)
{
    const uint8_t *s = (const uint8_t *)in;
    if (!in || !n_out || !dtype_out) return SZX_REF_ERR_INVALID;
    if (in_bytes < 64) return SZX_REF_ERR_CORRUPT;
    if (get_u32(s) != SZX_MAGIC || s[4] != SZX_VERSION) return SZX_REF_ERR_CORRUPT;
    const fmt_t *f = fmt_of(s[5]);
    uint32_t block = get_u32(s + 8);
    size_t G = get_u32(s + 12);
    size_t n = get_u64(s + 16);
    uint64_t total = get_u64(s + 56);
    if (!f || !block_ok(block) || n == 0) return SZX_REF_ERR_CORRUPT;
    if (G != tile_blocks_of(f, block)) return SZX_REF_ERR_CORRUPT;
    if (n > ((size_t)1 << 40) || total > in_bytes) return SZX_REF_ERR_CORRUPT;
    *n_out = n;
    *dtype_out = s[5];
    if (!out) return SZX_REF_ERR_INVALID;
    if (cap < n * (size_t)f->w) return SZX_REF_ERR_TOO_SMALL;

    geom_t g;
    geometry(f, n, block, G, &g);
    if (g.off_rec > total) return SZX_REF_ERR_CORRUPT;
    size_t rec_total = total - g.off_rec;
    if (get_u64(s + g.off_index + 8 * g.ntiles) != rec_total) return SZX_REF_ERR_CORRUPT;

    uint8_t *dst = (uint8_t *)out;
    uint64_t *t = (uint64_t *)malloc(block * sizeof(uint64_t));
    uint8_t *L = (uint8_t *)malloc(block);
    if (!t || !L) { free(t); free(L); return SZX_REF_ERR_INVALID; }
    int status = SZX_REF_OK;

    for (size_t tile = 0; tile < g.ntiles && status == SZX_REF_OK; tile++) {
        size_t k0 = tile * G, k1 = k0 + G < g.nb ? k0 + G : g.nb;
        uint64_t r0 = get_u64(s + g.off_index + 8 * tile);
        uint64_t r1 = get_u64(s + g.off_index + 8 * (tile + 1));
        if (r0 > r1 || r1 > rec_total || r0 % 16 || r1 % 16) { status = SZX_REF_ERR_CORRUPT; break; }
        const uint8_t *p = s + g.off_rec + r0;
        size_t size = r1 - r0;
        size_t nn_t = 0;
        for (size_t k = k0; k < k1; k++) nn_t += (s[g.off_state + k / 8] >> (k % 8)) & 1;
        size_t lead_bytes = nn_t * (block / 4);
        if (lead_bytes + nn_t > size) { status = SZX_REF_ERR_CORRUPT; break; }
        const uint8_t *lead = p, *reqs = p + lead_bytes;
        size_t cur = lead_bytes + nn_t; /* cursor into the record (mid bytes) */
        size_t rank = 0;
        for (size_t k = k0; k < k1 && status == SZX_REF_OK; k++) {
            size_t first = k * block;
            size_t len = first + block <= n ? block : n - first;
            uint64_t mu = load_value(f, s + g.off_mu + k * f->w);
            uint8_t *o = dst + first * f->w;
            if (!((s[g.off_state + k / 8] >> (k % 8)) & 1)) {
                for (size_t i = 0; i < len; i++) store_value(f, o + i * f->w, mu);
                continue;
            }
            const uint8_t *lc = lead + rank * (block / 4);
            int req = reqs[rank];
            rank++;
            if (req == 0xFF) {
                if (cur + len * f->w > size) { status = SZX_REF_ERR_CORRUPT; break; }
                memcpy(o, p + cur, len * f->w);
                cur += len * f->w;
                continue;
            }
            if (req < 1 + f->E || req > f->W) { status = SZX_REF_ERR_CORRUPT; break; }
            int sh = (8 - req % 8) % 8, q = (req + sh) / 8, lmax = q < 3 ? q : 3;
            for (size_t i = 0; i < block; i++) {
                int l = (lc[i >> 2] >> (2 * (i & 3))) & 3;
                if ((i >= len && l != 0) || l > lmax) status = SZX_REF_ERR_CORRUPT;
                L[i] = (uint8_t)l;
            }
            if (status != SZX_REF_OK) break;
            /* own bytes, plane by plane */
            for (size_t i = 0; i < len; i++) t[i] = 0;
            for (int j = 0; j < q && status == SZX_REF_OK; j++)
                for (size_t i = 0; i < len; i++)
                    if (L[i] <= j) {
                        if (cur >= size) { status = SZX_REF_ERR_CORRUPT; break; }
                        t[i] |= (uint64_t)p[cur++] << (f->W - 8 - 8 * j);
                    }
            if (status != SZX_REF_OK) break;
            /* leading bytes come from the previous value (t_{-1} = 0) */
            uint64_t prev = 0;
            for (size_t i = 0; i < len; i++) {
                for (int j = 0; j < L[i]; j++)
                    t[i] |= (uint64_t)byte_j(f, prev, j) << (f->W - 8 - 8 * j);
                prev = t[i];
                uint64_t vp = t[i] << sh;
                if (f->W == 32) vp &= 0xFFFFFFFFull;
                store_value(f, o + i * f->w, add_rn(f, vp, mu));
            }
        }
        if (status != SZX_REF_OK) break;
        if (rank != nn_t || pad16(cur) != size) { status = SZX_REF_ERR_CORRUPT; break; }
        for (size_t i = cur; i < size; i++)
            if (p[i] != 0) status = SZX_REF_ERR_CORRUPT;
    }
    free(t);
    free(L);
    return status;
}

/* ---- Eq. 6 diagnostics ---------------------------------------------------- */

int szx_ref_shift_overhead_bits(const void *in, size_t n, int dtype, double eb,
                                uint32_t block, uint64_t *bits_c,
                                uint64_t *bits_ab)
{
    const fmt_t *f = fmt_of(dtype);
    if (!f || !in || !bits_c || !bits_ab || n == 0 || !block_ok(block)) return SZX_REF_ERR_INVALID;
    if (!(eb > 0.0) || isinf(eb) || isnan(eb)) return SZX_REF_ERR_INVALID;
    uint64_t e = szx_ref_error_bound_bits(eb, dtype);
    const uint8_t *src = (const uint8_t *)in;
    uint8_t *lead = (uint8_t *)malloc(block / 4);
    uint8_t *mid = (uint8_t *)malloc(block * (size_t)f->w);
    uint64_t *work = (uint64_t *)malloc(2 * block * sizeof(uint64_t));
    if (!lead || !mid || !work) { free(lead); free(mid); free(work); return SZX_REF_ERR_INVALID; }
    *bits_c = 0;
    *bits_ab = 0;
    size_t nb = (n + block - 1) / block;
    for (size_t k = 0; k < nb; k++) {
        size_t first = k * block, len = first + block <= n ? block : n - first;
        const uint8_t *vals = src + first * f->w;
        block_out_t o;
        encode_block(f, vals, len, block, e, lead, mid, work, &o);
        if (o.kind != KIND_NONCONST) continue;
        /* Solution C: q - L_i bytes per value, L_i from the shifted words */
        int sh = (8 - o.req % 8) % 8, q = (o.req + sh) / 8;
        for (size_t i = 0; i < len; i++) {
            int l = (lead[i >> 2] >> (2 * (i & 3))) & 3;
            *bits_c += (uint64_t)(8 * (q - l));
        }
        /* Solutions A/B: the reqBits leading bits of v_i, unshifted, minus
         * their identical leading bytes against the previous value */
        uint64_t mu = o.mu, prev = 0;
        uint64_t keep = f->W == 64 ? ~(uint64_t)0 : 0xFFFFFFFFull;
        keep = (keep << (f->W - o.req)) & (f->W == 64 ? ~(uint64_t)0 : 0xFFFFFFFFull);
        for (size_t i = 0; i < len; i++) {
            uint64_t u = sub_rn(f, load_value(f, vals + i * f->w), mu) & keep;
            int l = lead_zero_bytes(f, u ^ prev);
            if (l > 3) l = 3;
            int bits = o.req - 8 * l;
            *bits_ab += (uint64_t)(bits > 0 ? bits : 0);
            prev = u;
        }
    }
    free(lead); free(mid); free(work);
    return SZX_REF_OK;
}
