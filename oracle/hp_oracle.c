/*
 * hp_oracle.c — sequential CPU oracle of the hierarchical loop-nest semantics.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the test suite, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py use it.  It shares no code, header
 * or constant with the CUDA library; the enumeration codes below are its own.
 *
 * What it computes (Sec. 2, recursive reduction "on each level, one of the
 * tasks collects the results from all sibling tasks"; Sec. 3.4 loop nests
 * bound to parallel levels): for a rectangular nest of depth d with extents
 * n_0..n_{d-1} and reduction level r,
 *
 *     out[i_0..i_{r-1}] = OP_{i_r < n_r} ... OP_{i_{d-1} < n_{d-1}} body(i_0..i_{d-1})
 *
 * and for a ragged (CSR) nest out[i] = OP_{e in [off[i], off[i+1])} body(i, e).
 * The result of any mapping of the levels onto hardware must equal this up to
 * floating-point rounding order; the oracle fixes the order to plain
 * lexicographic loop order and removes most rounding instead:
 *
 *   - FP32 inputs are widened to FP64; the product of two FP32 numbers is exact
 *     in FP64 (24 + 24 <= 53 significand bits).
 *   - FP64 sums use Neumaier's compensated summation (Neumaier 1974, "Rundungs-
 *     fehleranalyse einiger Verfahren zur Summation endlicher Summen"), error
 *     about 2 u64 |s| + O(n u64^2) sum|t|.
 *   - Integer work is exact in int64 with overflow detection.  For 32-bit
 *     integer nests body values and sums are reported modulo 2^32 (two's
 *     complement), which is what any wrapping 32-bit adder produces in any
 *     order; 64-bit nests widen int32 inputs and count overflowed outputs.
 *   - Every FP result is returned with sum|t| and sum t^2, so that errors can be
 *     stated per result against its conditioning.
 *
 * Build (done by oracle/__init__.py): gcc -O2 -std=c11 -fPIC -shared
 * -ffp-contract=off (no FMA contraction, which would change Neumaier's error
 * terms on Arm), no fast-math.
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>

/* oracle-private codes (the Python wrapper maps names onto these) */
enum { ORC_SUM = 0, ORC_MAX = 1, ORC_MIN = 2 };
enum { ORC_BODY_LOAD = 0, ORC_BODY_DOT_BCAST = 1, ORC_BODY_AFFINE = 3, ORC_BODY_GEOMETRIC = 4 };

#define ORC_MAX_DEPTH 8

/* Planted-mistake switch for the test suite's mutation checks; 0 (the only
 * value the oracle library is ever built with outside those checks) leaves
 * every formula as written.  1 drops the last term of each innermost loop,
 * 2 negates odd-indexed terms, 3 transposes the broadcast operand's index,
 * 4 drops the Neumaier compensation, 5 reduces one level too few,
 * 6 doubles sum|t|, 7 adds |t| instead of t^2 to sum t^2, 8 adds t instead of
 * |t| to sum|t|. */
#ifndef ORACLE_MUTATION
#define ORACLE_MUTATION 0
#endif

/* ------------------------------------------------------------------ */
/* FP64 accumulator: Neumaier sum, plus max/min, plus conditioning sums */
typedef struct {
    double sum, comp;      /* Neumaier running sum and running compensation */
    double best;           /* running max or min */
    double abs_sum;        /* sum |t| */
    double sq_sum;         /* sum t^2 */
    int64_t count;
} fp_acc;

static void fp_init(fp_acc *a, int op)
{
    a->sum = 0.0;
    a->comp = 0.0;
    a->best = (op == ORC_MAX) ? -INFINITY : INFINITY;
    a->abs_sum = 0.0;
    a->sq_sum = 0.0;
    a->count = 0;
}

static void fp_add(fp_acc *a, int op, double t)
{
    if (op == ORC_SUM) {
        double s = a->sum + t;
        if (ORACLE_MUTATION != 4) {
            if (fabs(a->sum) >= fabs(t))
                a->comp += (a->sum - s) + t;
            else
                a->comp += (t - s) + a->sum;
        }
        a->sum = s;
    } else if (op == ORC_MAX) {
        if (t > a->best) a->best = t;
    } else {
        if (t < a->best) a->best = t;
    }
    if (ORACLE_MUTATION == 6) a->abs_sum += 2.0 * fabs(t);
    else if (ORACLE_MUTATION == 8) a->abs_sum += t;
    else a->abs_sum += fabs(t);
    a->sq_sum += (ORACLE_MUTATION == 7) ? fabs(t) : t * t;
    a->count += 1;
}

static double fp_result(const fp_acc *a, int op)
{
    return (op == ORC_SUM) ? a->sum + a->comp : a->best;
}

/* int64 accumulator with overflow detection */
typedef struct {
    int64_t v;
    int overflow;
} int_acc;

static void int_init(int_acc *a, int op, int bits)
{
    a->overflow = 0;
    if (op == ORC_SUM) a->v = 0;
    else if (op == ORC_MAX) a->v = (bits == 32) ? (int64_t)INT32_MIN : INT64_MIN;
    else a->v = (bits == 32) ? (int64_t)INT32_MAX : INT64_MAX;
}

static void int_add(int_acc *a, int op, int64_t t)
{
    if (op == ORC_SUM) {
        int64_t s;
        if (__builtin_add_overflow(a->v, t, &s)) a->overflow = 1;
        a->v = s;
    } else if (op == ORC_MAX) {
        if (t > a->v) a->v = t;
    } else {
        if (t < a->v) a->v = t;
    }
}

/* a 32-bit wrapping adder yields the exact sum modulo 2^32 in any order */
static int64_t wrap32(int64_t v)
{
    uint32_t u = (uint32_t)(uint64_t)v;
    return (u & 0x80000000u) ? (int64_t)u - (int64_t)4294967296LL : (int64_t)u;
}

/* ------------------------------------------------------------------ */
/* bodies                                                               */
typedef struct {
    int depth, red_level, op, body, int_bits;
    const int64_t *ext;
    const float *Af, *wf;          /* FP inputs */
    const int32_t *Ai, *wi;        /* integer inputs */
    const double *params;          /* AFFINE: a, b, m ; GEOMETRIC: q, m */
} nest_ctx;

/* GEOMETRIC: value = fl32(q^(flat mod m)), q^k formed in FP64 by repeated
 * multiplication (exact for the dyadic q the tests use) */
static double geometric_term(double q, int64_t k)
{
    double v = 1.0;
    for (int64_t i = 0; i < k; ++i) v *= q;
    return (double)(float)v;
}

static int64_t mutated_rflat(const nest_ctx *c, int64_t rflat)
{
    /* mutation 3: read the broadcast operand as if its two innermost
     * reduced levels were swapped */
    if (ORACLE_MUTATION == 3 && c->depth - c->red_level >= 2) {
        int64_t n1 = c->ext[c->depth - 1], n0 = c->ext[c->depth - 2];
        int64_t k = rflat % n1, j = (rflat / n1) % n0, hi = rflat / (n1 * n0);
        return (hi * n1 + k) * n0 + j;
    }
    return rflat;
}

static double mutated_sign(int64_t flat)
{
    return (ORACLE_MUTATION == 2 && (flat & 1)) ? -1.0 : 1.0;
}

static double body_fp_exact(const nest_ctx *c, int64_t flat, int64_t rflat);

static double body_fp(const nest_ctx *c, int64_t flat, int64_t rflat)
{
    return mutated_sign(flat) * body_fp_exact(c, flat, mutated_rflat(c, rflat));
}

static double body_fp_exact(const nest_ctx *c, int64_t flat, int64_t rflat)
{
    switch (c->body) {
    case ORC_BODY_LOAD:
        return (double)c->Af[flat];
    case ORC_BODY_DOT_BCAST:
        return (double)c->Af[flat] * (double)c->wf[rflat];
    case ORC_BODY_AFFINE: {
        int64_t m = (int64_t)c->params[2];
        return c->params[0] + c->params[1] * (double)(flat % m);
    }
    default: {
        int64_t m = (int64_t)c->params[1];
        return geometric_term(c->params[0], flat % m);
    }
    }
}

static int64_t body_int_exact(const nest_ctx *c, int64_t flat, int64_t rflat);

static int64_t wrap32(int64_t v);

/* 32-bit integer nests compute body values modulo 2^32 as well */
static int64_t body_int(const nest_ctx *c, int64_t flat, int64_t rflat)
{
    int64_t v = (int64_t)mutated_sign(flat) * body_int_exact(c, flat, mutated_rflat(c, rflat));
    return (c->int_bits == 32) ? wrap32(v) : v;
}

static int64_t body_int_exact(const nest_ctx *c, int64_t flat, int64_t rflat)
{
    switch (c->body) {
    case ORC_BODY_LOAD:
        return (int64_t)c->Ai[flat];
    case ORC_BODY_DOT_BCAST:
        return (int64_t)c->Ai[flat] * (int64_t)c->wi[rflat];
    default: {
        int64_t a = (int64_t)c->params[0], b = (int64_t)c->params[1], m = (int64_t)c->params[2];
        return a + b * (flat % m);
    }
    }
}

/* ------------------------------------------------------------------ */
/* recursive formulation: loops in lexicographic order                  */
static void visit_reduced_fp(const nest_ctx *c, int l, int64_t flat, int64_t rflat, fp_acc *acc)
{
    if (l == c->depth) {
        fp_add(acc, c->op, body_fp(c, flat, rflat));
        return;
    }
    int64_t n = c->ext[l];
    if (ORACLE_MUTATION == 1 && l == c->depth - 1 && n > 0) n -= 1;
    for (int64_t i = 0; i < n; ++i)
        visit_reduced_fp(c, l + 1, flat * c->ext[l] + i, rflat * c->ext[l] + i, acc);
}

static void visit_reduced_int(const nest_ctx *c, int l, int64_t flat, int64_t rflat, int_acc *acc)
{
    if (l == c->depth) {
        int_add(acc, c->op, body_int(c, flat, rflat));
        return;
    }
    int64_t n = c->ext[l];
    if (ORACLE_MUTATION == 1 && l == c->depth - 1 && n > 0) n -= 1;
    for (int64_t i = 0; i < n; ++i)
        visit_reduced_int(c, l + 1, flat * c->ext[l] + i, rflat * c->ext[l] + i, acc);
}

typedef struct {
    double *out_fp, *abs_sum, *sq_sum;
    int64_t *out_int;
    int64_t overflow_count;
} sink;

static void emit_fp(const nest_ctx *c, sink *s, int64_t oidx, const fp_acc *acc)
{
    s->out_fp[oidx] = fp_result(acc, c->op);
    if (s->abs_sum) s->abs_sum[oidx] = acc->abs_sum;
    if (s->sq_sum) s->sq_sum[oidx] = acc->sq_sum;
}

static void emit_int(const nest_ctx *c, sink *s, int64_t oidx, const int_acc *acc)
{
    int64_t v = acc->v;
    if (c->int_bits == 32 && c->op == ORC_SUM) v = wrap32(v);
    else if (acc->overflow) s->overflow_count += 1;
    s->out_int[oidx] = v;
}

static void visit_outputs(const nest_ctx *c, sink *s, int l, int64_t flat, int64_t oidx)
{
    int start = c->red_level;
    if (ORACLE_MUTATION == 5 && start < c->depth) start += 1;   /* reduces one level too few */
    if (l == start) {
        if (start != c->red_level) oidx /= c->ext[c->red_level];
        if (c->int_bits) {
            int_acc acc;
            int_init(&acc, c->op, c->int_bits);
            visit_reduced_int(c, l, flat, 0, &acc);
            emit_int(c, s, oidx, &acc);
        } else {
            fp_acc acc;
            fp_init(&acc, c->op);
            visit_reduced_fp(c, l, flat, 0, &acc);
            emit_fp(c, s, oidx, &acc);
        }
        return;
    }
    for (int64_t i = 0; i < c->ext[l]; ++i)
        visit_outputs(c, s, l + 1, flat * c->ext[l] + i, oidx * c->ext[l] + i);
}

static int check_args(int depth, const int64_t *ext, int red_level, int op)
{
    if (depth < 1 || depth > ORC_MAX_DEPTH) return -1;
    if (red_level < 0 || red_level > depth) return -1;
    if (op < ORC_SUM || op > ORC_MIN) return -1;
    for (int l = 0; l < depth; ++l)
        if (ext[l] < 0) return -1;
    return 0;
}

/*
 * Rectangular nest, full evaluation.  int_bits = 0 selects the FP path
 * (inputs Af/wf), 32 or 64 the integer path (inputs Ai/wi, int32).
 * Outputs are row-major over levels 0..red_level-1.
 * Returns -1 on bad arguments, else the number of int64 outputs whose exact
 * value overflowed (always 0 for the FP path and for 32-bit sums).
 */
int64_t oracle_rect(int depth, const int64_t *ext, int red_level, int op, int body, int int_bits,
                    const float *Af, const float *wf, const int32_t *Ai, const int32_t *wi,
                    const double *params, double *out_fp, int64_t *out_int,
                    double *abs_sum, double *sq_sum)
{
    if (check_args(depth, ext, red_level, op)) return -1;
    nest_ctx c = {depth, red_level, op, body, int_bits, ext, Af, wf, Ai, wi, params};
    sink s = {out_fp, abs_sum, sq_sum, out_int, 0};
    visit_outputs(&c, &s, 0, 0, 0);
    return s.overflow_count;
}

/*
 * Rectangular nest, selected outputs only (full-size parity on samples).
 * oidx[k] is a row-major output index; results go to slot k.
 */
int64_t oracle_rect_sampled(int depth, const int64_t *ext, int red_level, int op, int body, int int_bits,
                            const float *Af, const float *wf, const int32_t *Ai, const int32_t *wi,
                            const double *params, const int64_t *oidx, int64_t n_samples,
                            double *out_fp, int64_t *out_int, double *abs_sum, double *sq_sum)
{
    if (check_args(depth, ext, red_level, op)) return -1;
    nest_ctx c = {depth, red_level, op, body, int_bits, ext, Af, wf, Ai, wi, params};
    sink s = {out_fp, abs_sum, sq_sum, out_int, 0};
    int64_t n_out = 1;
    for (int l = 0; l < red_level; ++l) n_out *= ext[l];
    for (int64_t k = 0; k < n_samples; ++k) {
        if (oidx[k] < 0 || oidx[k] >= n_out) return -1;
        /* the flat prefix of output o over levels 0..r-1 is o itself */
        if (int_bits) {
            int_acc acc;
            int_init(&acc, op, int_bits);
            visit_reduced_int(&c, red_level, oidx[k], 0, &acc);
            emit_int(&c, &s, k, &acc);
        } else {
            fp_acc acc;
            fp_init(&acc, op);
            visit_reduced_fp(&c, red_level, oidx[k], 0, &acc);
            emit_fp(&c, &s, k, &acc);
        }
    }
    return s.overflow_count;
}

/*
 * Second, independent formulation: one flat loop over the whole iteration
 * space; each flat index f is split into its output part f / R and its
 * reduced part f % R (mixed radix, row-major).  Same per-output visiting order
 * as the recursive form, so results must agree bit for bit.
 */
int64_t oracle_rect_flat(int depth, const int64_t *ext, int red_level, int op, int body, int int_bits,
                         const float *Af, const float *wf, const int32_t *Ai, const int32_t *wi,
                         const double *params, double *out_fp, int64_t *out_int,
                         double *abs_sum, double *sq_sum, void *scratch)
{
    if (check_args(depth, ext, red_level, op)) return -1;
    nest_ctx c = {depth, red_level, op, body, int_bits, ext, Af, wf, Ai, wi, params};
    int64_t n_out = 1, n_red = 1;
    for (int l = 0; l < red_level; ++l) n_out *= ext[l];
    for (int l = red_level; l < depth; ++l) n_red *= ext[l];
    fp_acc *fa = (fp_acc *)scratch;     /* caller provides n_out accumulators */
    int_acc *ia = (int_acc *)scratch;
    for (int64_t o = 0; o < n_out; ++o) {
        if (int_bits) int_init(&ia[o], op, int_bits);
        else fp_init(&fa[o], op);
    }
    int64_t total = n_out * n_red;
    for (int64_t f = 0; f < total; ++f) {
        int64_t o = f / n_red, rho = f % n_red;
        if (int_bits) int_add(&ia[o], op, body_int(&c, f, rho));
        else fp_add(&fa[o], op, body_fp(&c, f, rho));
    }
    sink s = {out_fp, abs_sum, sq_sum, out_int, 0};
    for (int64_t o = 0; o < n_out; ++o) {
        if (int_bits) emit_int(&c, &s, o, &ia[o]);
        else emit_fp(&c, &s, o, &fa[o]);
    }
    return s.overflow_count;
}

/* size in bytes of the scratch oracle_rect_flat needs per output */
int64_t oracle_flat_scratch_per_output(void)
{
    return (int64_t)(sizeof(fp_acc) > sizeof(int_acc) ? sizeof(fp_acc) : sizeof(int_acc));
}

/*
 * Ragged nest in CSR form, FP body val[e] * x[col[e]] (Sec. 3.8 partitions a
 * level into uneven pieces; this is the ragged inner loop itself).
 * rows: list of row ids to evaluate (NULL = all rows, in order).
 */
int oracle_csr(int64_t n_rows, const int64_t *off, const int32_t *col, const float *val,
               const float *x, int64_t n_x, int op, const int64_t *rows, int64_t n_eval,
               double *out, double *abs_sum, double *sq_sum)
{
    if (op < ORC_SUM || op > ORC_MIN || n_rows < 0) return -1;
    int64_t n = rows ? n_eval : n_rows;
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = rows ? rows[k] : k;
        if (i < 0 || i >= n_rows || off[i] > off[i + 1]) return -1;
        fp_acc acc;
        fp_init(&acc, op);
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            if (col[e] < 0 || (int64_t)col[e] >= n_x) return -1;
            fp_add(&acc, op, (double)val[e] * (double)x[col[e]]);
        }
        out[k] = fp_result(&acc, op);
        if (abs_sum) abs_sum[k] = acc.abs_sum;
        if (sq_sum) sq_sum[k] = acc.sq_sum;
    }
    return 0;
}

/*
 * Count histogram over the entries of a CSR nest: hist[b] = #{e : col[e] >> shift == b}.
 * Returns the number of entries whose bin falls outside [0, n_bins) (not counted).
 */
int64_t oracle_hist(int64_t nnz, const int32_t *col, int shift, int64_t n_bins, int64_t *hist)
{
    int64_t outside = 0;
    for (int64_t b = 0; b < n_bins; ++b) hist[b] = 0;
    for (int64_t e = 0; e < nnz; ++e) {
        int64_t v = (int64_t)col[e];
        int64_t b = (v >= 0) ? (v >> shift) : -1;
        if (b < 0 || b >= n_bins) outside += 1;
        else hist[b] += 1;
    }
    return outside;
}
