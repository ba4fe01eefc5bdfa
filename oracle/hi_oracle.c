/*
 * hi_oracle.c -- plain, slow CPU oracle for the interpolation predictor +
 * error-bounded linear quantizer of cuSZ-Hi (arXiv 2507.11165).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the timed CPU baseline
 * of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * What it follows (paper sections):
 *   Sec. 3.1, Eq. 1      -- the pointwise bound |x - x'| <= eps.
 *   Sec. 3.2             -- anchor grid stored losslessly, hierarchical
 *                           interpolation from large to small stride, one
 *                           independent data block per thread block.
 *   Sec. 5.1.1           -- (A+1)^d blocks that include their anchors,
 *                           anchor stride A (16 in the paper), log2(A) levels.
 *   Sec. 5.1.2           -- 1D interpolation passes along a dimension
 *                           sequence; linear / quadratic / cubic splines.
 *   Sec. 5.1.3           -- auto-tuning on uniformly sampled blocks (0.2 %)
 *                           with per-level minimum aggregated error.
 *   Sec. 5.2.1           -- one-byte quantization codes, outliers stored
 *                           separately; Sec. 5.2.3: 128 is the zero symbol.
 *   Sec. 6.1.4 (metrics) -- value-range-relative error bound.
 *
 * Readings where the paper is silent (the same list is kept with the design
 * notes of the repository):
 *   - stencil weights are the Lagrange midpoint weights: linear (1,1)/2,
 *     cubic (-1,9,9,-1)/16, and the two one-sided quadratics (3,6,-1)/8 and
 *     (-1,6,3)/8 near a block edge; a point with no right neighbour (only at
 *     the global upper edge) is extrapolated linearly, (3b - a)/2, or copied;
 *   - stencils never leave their block (blocks are independent);
 *   - quantization radius R = 128: q in [-127,127] maps to code q+128,
 *     code 0 marks an outlier;  t = (x-p)*r with r = fl(1/(2 eps)), q =
 *     rint(t) (ties to even), x' = p + q*fl(2 eps);  outlier when
 *     !(|t| < 127.5) or !(|x - x'| < eb_f), eb_f = largest float <= eps;
 *   - value-range-relative bound: eps = eb * (max - min) over finite values,
 *     eps = eb for a constant field;
 *   - auto-tune error = sum of |x - p| with predictions taken from the
 *     original (not reconstructed) values; ties go to the first config in
 *     enumeration order (cubic before linear, lexicographic permutations).
 *
 * Arithmetic: float32, every operation written out in the order it is
 * evaluated; build with -ffp-contract=off and without fast-math so no
 * multiply-add is ever contracted.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ETRAVERSAL 10 /* a stencil point was read before it was known  */
#define ORC_EREVISIT 11   /* a point was predicted twice inside one block   */
#define ORC_EMISSED 12    /* a point of a block was never predicted         */
#define ORC_EFACE 13      /* two blocks disagree on a shared face point      */
#define ORC_ECORRUPT 14   /* decompress input references a missing outlier  */

#define ORC_LINEAR 0
#define ORC_CUBIC 1
#define ORC_MD_LINEAR 2 /* multi-dimensional interpolation, linear splines */
#define ORC_MD_CUBIC 3  /* multi-dimensional interpolation, cubic splines  */
#define ORC_RADIUS 128
#define ORC_MAX_LEVELS 8

/* ------------------------------------------------------------------------ */
/* Geometry: blocks of (A+1)^d points sharing their faces (Sec. 5.1.1).     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n[3];  /* field dims, slowest -> fastest; a dim of size 1 is inactive */
    int A;         /* anchor stride                                           */
    int L;         /* number of interpolation levels, log2(A)                 */
    int64_t nb[3]; /* blocks per dim                                          */
    int64_t na[3]; /* anchors per dim                                         */
    int64_t N;     /* number of points                                        */
} geom;

static int ilog2_exact(int A)
{
    int l = 0;
    if (A < 2) return -1;
    while ((1 << l) < A) l++;
    return ((1 << l) == A) ? l : -1;
}

static int geom_init(geom* G, const int64_t dims[3], int A)
{
    int d;
    G->A = A;
    G->L = ilog2_exact(A);
    if (G->L < 1 || G->L > 5) return ORC_EINVAL;
    G->N = 1;
    for (d = 0; d < 3; d++) {
        if (dims[d] < 1) return ORC_EINVAL;
        G->n[d] = dims[d];
        G->N *= dims[d];
        if (dims[d] == 1) {
            G->nb[d] = 1;
        } else {
            G->nb[d] = (dims[d] - 1 + A - 1) / A; /* ceil((n-1)/A) */
        }
        G->na[d] = (dims[d] - 1) / A + 1;
    }
    return ORC_OK;
}

static int64_t gindex(const geom* G, int64_t g0, int64_t g1, int64_t g2)
{
    return (g0 * G->n[1] + g1) * G->n[2] + g2;
}

static int is_anchor(const geom* G, int64_t g0, int64_t g1, int64_t g2)
{
    return (g0 % G->A == 0) && (g1 % G->A == 0) && (g2 % G->A == 0);
}

/* ------------------------------------------------------------------------ */
/* Error-bound constants (Eq. 1 and the value-range-relative bound).       */
/* ------------------------------------------------------------------------ */
int hi_oracle_eps(int eb_mode, double eb, const float* x, int64_t N, float* out5, double* eps_out)
{
    int64_t i;
    int any = 0;
    float vmin = INFINITY, vmax = -INFINITY;
    double eps;
    float eb_f, ebx2_f, r_f;

    if (!(eb > 0.0) || !isfinite(eb) || (eb_mode != 0 && eb_mode != 1) || N < 0) return ORC_EINVAL;
    for (i = 0; i < N; i++) {
        float v = x[i];
        if (!isfinite(v)) continue;
        if (!any) {
            vmin = v;
            vmax = v;
            any = 1;
        } else {
            if (v < vmin) vmin = v;
            if (v > vmax) vmax = v;
        }
    }
    if (!any) {
        vmin = 0.0f;
        vmax = 0.0f;
    }
    /* a signed zero is reported as +0 */
    vmin = vmin + 0.0f;
    vmax = vmax + 0.0f;

    if (eb_mode == 0) {
        eps = eb;
    } else {
        double range = (double)vmax - (double)vmin;
        eps = (range > 0.0) ? eb * range : eb;
    }
    if (!(eps > 0.0) || !isfinite(eps)) return ORC_EINVAL;

    /* eb_f: the largest float not above eps */
    eb_f = (float)eps;
    if ((double)eb_f > eps) eb_f = nextafterf(eb_f, 0.0f);
    ebx2_f = (float)(2.0 * eps);
    r_f = (float)(1.0 / (2.0 * eps));
    if (!(eb_f > 0.0f) || !isfinite(ebx2_f) || !isfinite(r_f) || !(r_f > 0.0f)) return ORC_EINVAL;

    out5[0] = eb_f;
    out5[1] = ebx2_f;
    out5[2] = r_f;
    out5[3] = vmin;
    out5[4] = vmax;
    if (eps_out) *eps_out = eps;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Prediction along one line (Sec. 5.1.2; weights: reading above).          */
/* a = f(c-3s), b = f(c-s), u = f(c+s), v = f(c+3s)                         */
/* ------------------------------------------------------------------------ */
static float predict_line(int interp, int have_l3, int have_r, int have_r3, float a, float b, float u,
                          float v)
{
    if (!have_r) {
        /* global upper edge: no point at c+s */
        if (have_l3) return (3.0f * b - a) * 0.5f;
        return b;
    }
    if (interp == ORC_LINEAR) return (b + u) * 0.5f;
    if (have_l3 && have_r3) return (9.0f * (b + u) - (a + v)) * 0.0625f;
    if (have_r3) return ((3.0f * b + 6.0f * u) - v) * 0.125f;
    if (have_l3) return ((6.0f * b + 3.0f * u) - a) * 0.125f;
    return (b + u) * 0.5f;
}

/* Which stencil predict_line uses (for the traversal trace):
 * 0 linear midpoint, 1 cubic 4-point, 2 quadratic without f(c-3s),
 * 3 quadratic without f(c+3s), 4 linear extrapolation, 5 copy of f(c-s). */
static int stencil_case(int interp, int have_l3, int have_r, int have_r3)
{
    if (!have_r) return have_l3 ? 4 : 5;
    if (interp == ORC_LINEAR) return 0;
    if (have_l3 && have_r3) return 1;
    if (have_r3) return 2;
    if (have_l3) return 3;
    return 0;
}

/* Order of the stencil predict_line uses, for the multi-dimensional scheme's
 * "highest spline order" rule: 3 cubic, 2 quadratic, 1 linear (midpoint or
 * extrapolation), 0 copy. */
static int stencil_order(int interp, int have_l3, int have_r, int have_r3)
{
    if (!have_r) return have_l3 ? 1 : 0;
    if (interp == ORC_LINEAR) return 1;
    if (have_l3 && have_r3) return 3;
    if (have_l3 || have_r3) return 2;
    return 1;
}

/* Linear quantization of the prediction error (Sec. 5.2.1).  Returns the
 * code (1..255, or 0 for an outlier) and stores the reconstructed value. */
static int quantize(float x, float p, float eb_f, float ebx2_f, float r_f, float* xr_out)
{
    float t = (x - p) * r_f;
    float qf, xr;
    if (!(fabsf(t) < 127.5f)) {
        *xr_out = x;
        return 0;
    }
    qf = rintf(t);
    xr = p + qf * ebx2_f;
    if (!(fabsf(x - xr) < eb_f)) {
        *xr_out = x;
        return 0;
    }
    *xr_out = xr;
    return (int)qf + ORC_RADIUS;
}

/* ------------------------------------------------------------------------ */
/* One block.                                                               */
/* ------------------------------------------------------------------------ */
enum { MODE_COMPRESS = 0, MODE_DECOMPRESS = 1, MODE_TUNE = 2 };

typedef struct {
    const geom* G;
    int64_t o[3]; /* origin */
    int e[3];     /* local extent per dim (0 for an inactive dim) */
    int P;        /* local pitch: A+1 */
    float* orig;  /* original values (compress, tune) */
    float* rec;   /* reconstructed values */
    uint8_t* known;
    uint8_t* code;
} block;

static int lidx(const block* B, int c0, int c1, int c2)
{
    return (c0 * B->P + c1) * B->P + c2;
}

static void block_init(block* B, const geom* G, int64_t t0, int64_t t1, int64_t t2)
{
    int64_t t[3];
    int d;
    t[0] = t0;
    t[1] = t1;
    t[2] = t2;
    B->G = G;
    B->P = G->A + 1;
    for (d = 0; d < 3; d++) {
        B->o[d] = t[d] * G->A;
        if (G->n[d] == 1) {
            B->e[d] = 0;
        } else {
            int64_t rem = G->n[d] - 1 - B->o[d];
            B->e[d] = (int)(rem < G->A ? rem : G->A);
        }
    }
    memset(B->known, 0, (size_t)B->P * B->P * B->P);
}

typedef struct {
    int mode;
    float eb_f, ebx2_f, r_f;
    /* decompress inputs */
    const uint8_t* g_codes;
    const float* g_outval; /* dense outlier values, indexed by point */
    const uint8_t* g_outhas;
    /* tune output */
    double err;
    /* optional traversal trace, indexed by point: level, dimension, stencil case */
    int8_t* t_lvl;
    int8_t* t_dir;
    int8_t* t_case;
    int status;
} action;

/* The prediction pr of point c (local index li) is final: quantize it
 * (compress), rebuild from the code (decompress) or add |x - pr| (tune), and
 * record the trace; the point becomes known. */
static void apply_point(block* B, const int c[3], int li, float pr, int l, int dir, int kc, action* act)
{
    if (act->mode == MODE_COMPRESS) {
        float xr;
        int k = quantize(B->orig[li], pr, act->eb_f, act->ebx2_f, act->r_f, &xr);
        B->code[li] = (uint8_t)k;
        B->rec[li] = xr;
    } else if (act->mode == MODE_DECOMPRESS) {
        int64_t g = gindex(B->G, B->o[0] + c[0], B->o[1] + c[1], B->o[2] + c[2]);
        int k = act->g_codes[g];
        B->code[li] = (uint8_t)k;
        if (k == 0) {
            if (!act->g_outhas[g]) {
                act->status = ORC_ECORRUPT;
                return;
            }
            B->rec[li] = act->g_outval[g];
        } else {
            B->rec[li] = pr + (float)(k - ORC_RADIUS) * act->ebx2_f;
        }
    } else {
        float x = B->orig[li];
        act->err += (double)fabsf(x - pr);
    }
    if (act->t_lvl) {
        int64_t g = gindex(B->G, B->o[0] + c[0], B->o[1] + c[1], B->o[2] + c[2]);
        if (act->t_lvl[g] >= 0 && (act->t_lvl[g] != l || act->t_dir[g] != dir || act->t_case[g] != kc)) {
            act->status = ORC_EFACE;
            return;
        }
        act->t_lvl[g] = (int8_t)l;
        act->t_dir[g] = (int8_t)dir;
        act->t_case[g] = (int8_t)kc;
    }
    B->known[li] = 1;
}

/* The 1D stencil of point c along dim d at stride s: availability, the
 * known-before-use check, the values (from `src`) and the prediction.
 * Returns 0, or ORC_ETRAVERSAL. */
static int line_predict(const block* B, const float* src, const int c[3], int d, int s, int interp, float* pr,
                        int* kc, int* ord)
{
    int cd = c[d], e = B->e[d];
    int have_l3 = (cd - 3 * s) >= 0;
    int have_r = (cd + s) <= e;
    int have_r3 = (cd + 3 * s) <= e;
    int cm[3];
    float a = 0.0f, b, u = 0.0f, v = 0.0f;
    int lb, la = -1, lu = -1, lv = -1;
    memcpy(cm, c, sizeof cm);
    cm[d] = cd - s;
    lb = lidx(B, cm[0], cm[1], cm[2]);
    if (have_r) {
        cm[d] = cd + s;
        lu = lidx(B, cm[0], cm[1], cm[2]);
    }
    if (have_l3) {
        cm[d] = cd - 3 * s;
        la = lidx(B, cm[0], cm[1], cm[2]);
    }
    if (have_r3) {
        cm[d] = cd + 3 * s;
        lv = lidx(B, cm[0], cm[1], cm[2]);
    }
    if (!B->known[lb] || (lu >= 0 && !B->known[lu]) || (la >= 0 && !B->known[la]) || (lv >= 0 && !B->known[lv]))
        return ORC_ETRAVERSAL;
    b = src[lb];
    if (lu >= 0) u = src[lu];
    if (la >= 0) a = src[la];
    if (lv >= 0) v = src[lv];
    *pr = predict_line(interp, have_l3, have_r, have_r3, a, b, u, v);
    *kc = stencil_case(interp, have_l3, have_r, have_r3);
    *ord = stencil_order(interp, have_l3, have_r, have_r3);
    return ORC_OK;
}

/* Multi-dimensional interpolation of level l (Sec. 5.1.2, parallelized
 * multi-dimensional interpolation; reading in the design notes): the level's
 * points, those whose coordinates are all multiples of s with at least one
 * odd multiple, are taken in three phases by the number k of odd-multiple
 * coordinates (1, then 2, then 3).  A point is interpolated along each of
 * its k odd dims with that dim's 1D stencil (the same cases as the 1D
 * scheme); only the interpolations of the highest order among them count,
 * and the prediction is their mean, summed in increasing dim order
 * (one: itself; two: sum * 0.5; three: sum / 3).  Its stencil nodes have
 * k - 1 odd coordinates, so they are known from the phase before. */
static void run_level_md(block* B, int l, int interp, action* act)
{
    int s = 1 << l;
    int k, d, c[3];
    const float* src = (act->mode == MODE_TUNE) ? B->orig : B->rec;
    for (k = 1; k <= 3; k++) {
        for (c[0] = 0; c[0] <= B->e[0]; c[0] += s)
            for (c[1] = 0; c[1] <= B->e[1]; c[1] += s)
                for (c[2] = 0; c[2] <= B->e[2]; c[2] += s) {
                    float p[3], pr, sum = 0.0f;
                    int ord[3], kc[3], odd[3], nodd = 0, best = -1, n = 0, mask = 0, li;
                    for (d = 0; d < 3; d++)
                        if (c[d] % (2 * s) == s) odd[nodd++] = d;
                    if (nodd != k) continue;
                    li = lidx(B, c[0], c[1], c[2]);
                    if (B->known[li]) {
                        act->status = ORC_EREVISIT;
                        return;
                    }
                    for (d = 0; d < nodd; d++) {
                        if (line_predict(B, src, c, odd[d], s, interp, &p[d], &kc[d], &ord[d])) {
                            act->status = ORC_ETRAVERSAL;
                            return;
                        }
                        if (ord[d] > best) best = ord[d];
                    }
                    for (d = 0; d < nodd; d++)
                        if (ord[d] == best) {
                            sum = (n == 0) ? p[d] : sum + p[d];
                            mask |= 1 << odd[d];
                            n++;
                        }
                    if (n == 1)
                        pr = sum;
                    else if (n == 2)
                        pr = sum * 0.5f;
                    else
                        pr = sum / 3.0f;
                    /* trace: dir = 3 + the mask of the averaged dims, case = their order */
                    apply_point(B, c, li, pr, l, 3 + mask, best, act);
                    if (act->status) return;
                }
    }
}

/* Every point c of the block with
 *   c[d_p] = s mod 2s,  c[d_q] = 0 mod s (q < p),  c[d_q] = 0 mod 2s (q > p)
 * is predicted in pass p of level l (stride s = 2^l) along d_p = order[p]. */
static void run_level(block* B, int l, int interp, const uint8_t order[3], action* act)
{
    int s = 1 << l;
    int p, q, d;
    for (p = 0; p < 3; p++) {
        int dp = order[p];
        int start[3], step[3];
        int c[3];
        for (q = 0; q < 3; q++) {
            d = order[q];
            if (q == p) {
                start[d] = s;
                step[d] = 2 * s;
            } else if (q < p) {
                start[d] = 0;
                step[d] = s;
            } else {
                start[d] = 0;
                step[d] = 2 * s;
            }
        }
        for (c[0] = start[0]; c[0] <= B->e[0]; c[0] += step[0])
            for (c[1] = start[1]; c[1] <= B->e[1]; c[1] += step[1])
                for (c[2] = start[2]; c[2] <= B->e[2]; c[2] += step[2]) {
                    int li = lidx(B, c[0], c[1], c[2]);
                    int cd = c[dp];
                    int e = B->e[dp];
                    int have_l3 = (cd - 3 * s) >= 0;
                    int have_r = (cd + s) <= e;
                    int have_r3 = (cd + 3 * s) <= e;
                    int cm[3], cl[3];
                    float a = 0.0f, b, u = 0.0f, v = 0.0f, pr;
                    const float* src = (act->mode == MODE_TUNE) ? B->orig : B->rec;
                    int lb, la = -1, lu = -1, lv = -1;

                    if (B->known[li]) {
                        act->status = ORC_EREVISIT;
                        return;
                    }
                    memcpy(cm, c, sizeof cm);
                    memcpy(cl, c, sizeof cl);
                    cm[dp] = cd - s;
                    lb = lidx(B, cm[0], cm[1], cm[2]);
                    if (have_r) {
                        cm[dp] = cd + s;
                        lu = lidx(B, cm[0], cm[1], cm[2]);
                    }
                    if (have_l3) {
                        cl[dp] = cd - 3 * s;
                        la = lidx(B, cl[0], cl[1], cl[2]);
                    }
                    if (have_r3) {
                        cl[dp] = cd + 3 * s;
                        lv = lidx(B, cl[0], cl[1], cl[2]);
                    }
                    /* every stencil point must already be known */
                    if (!B->known[lb] || (lu >= 0 && !B->known[lu]) || (la >= 0 && !B->known[la]) ||
                        (lv >= 0 && !B->known[lv])) {
                        act->status = ORC_ETRAVERSAL;
                        return;
                    }
                    b = src[lb];
                    if (lu >= 0) u = src[lu];
                    if (la >= 0) a = src[la];
                    if (lv >= 0) v = src[lv];
                    pr = predict_line(interp, have_l3, have_r, have_r3, a, b, u, v);

                    if (act->mode == MODE_COMPRESS) {
                        float xr;
                        int k = quantize(B->orig[li], pr, act->eb_f, act->ebx2_f, act->r_f, &xr);
                        B->code[li] = (uint8_t)k;
                        B->rec[li] = xr;
                    } else if (act->mode == MODE_DECOMPRESS) {
                        int64_t g = gindex(B->G, B->o[0] + c[0], B->o[1] + c[1], B->o[2] + c[2]);
                        int k = act->g_codes[g];
                        B->code[li] = (uint8_t)k;
                        if (k == 0) {
                            if (!act->g_outhas[g]) {
                                act->status = ORC_ECORRUPT;
                                return;
                            }
                            B->rec[li] = act->g_outval[g];
                        } else {
                            B->rec[li] = pr + (float)(k - ORC_RADIUS) * act->ebx2_f;
                        }
                    } else {
                        float x = B->orig[li];
                        act->err += (double)fabsf(x - pr);
                    }
                    if (act->t_lvl) {
                        int64_t g = gindex(B->G, B->o[0] + c[0], B->o[1] + c[1], B->o[2] + c[2]);
                        int kc = stencil_case(interp, have_l3, have_r, have_r3);
                        if (act->t_lvl[g] >= 0 &&
                            (act->t_lvl[g] != l || act->t_dir[g] != dp || act->t_case[g] != kc)) {
                            act->status = ORC_EFACE;
                            return;
                        }
                        act->t_lvl[g] = (int8_t)l;
                        act->t_dir[g] = (int8_t)dp;
                        act->t_case[g] = (int8_t)kc;
                    }
                    B->known[li] = 1;
                }
    }
}

/* Seed the anchors of a block; load originals if needed. */
static void block_seed(block* B, const float* x, const float* anchors, int mode)
{
    const geom* G = B->G;
    int c0, c1, c2;
    for (c0 = 0; c0 <= B->e[0]; c0++)
        for (c1 = 0; c1 <= B->e[1]; c1++)
            for (c2 = 0; c2 <= B->e[2]; c2++) {
                int li = lidx(B, c0, c1, c2);
                int64_t g0 = B->o[0] + c0, g1 = B->o[1] + c1, g2 = B->o[2] + c2;
                if (mode != MODE_DECOMPRESS) B->orig[li] = x[gindex(G, g0, g1, g2)];
                if (is_anchor(G, g0, g1, g2)) {
                    float av;
                    if (mode == MODE_DECOMPRESS) {
                        av = anchors[(g0 / G->A * G->na[1] + g1 / G->A) * G->na[2] + g2 / G->A];
                    } else {
                        av = x[gindex(G, g0, g1, g2)];
                    }
                    B->rec[li] = av;
                    B->code[li] = ORC_RADIUS;
                    B->known[li] = 1;
                }
            }
}

static int block_complete(const block* B)
{
    int c0, c1, c2;
    for (c0 = 0; c0 <= B->e[0]; c0++)
        for (c1 = 0; c1 <= B->e[1]; c1++)
            for (c2 = 0; c2 <= B->e[2]; c2++)
                if (!B->known[lidx(B, c0, c1, c2)]) return 0;
    return 1;
}

static int check_levels(int L, const uint8_t* interp, const uint8_t* order)
{
    int l;
    for (l = 0; l < L; l++) {
        int seen = 0, q;
        if (interp[l] > ORC_MD_CUBIC) return ORC_EINVAL;
        for (q = 0; q < 3; q++) {
            if (order[3 * l + q] > 2) return ORC_EINVAL;
            seen |= 1 << order[3 * l + q];
        }
        if (seen != 7) return ORC_EINVAL;
    }
    return ORC_OK;
}

/* Run every level of one block, from the coarsest to the finest. */
/* One level under its configuration: the 1D dimension sequence, or the
 * multi-dimensional scheme (with linear or cubic splines). */
static void run_level_any(block* B, int l, int interp, const uint8_t order[3], action* act)
{
    if (interp == ORC_MD_LINEAR || interp == ORC_MD_CUBIC)
        run_level_md(B, l, interp == ORC_MD_CUBIC ? ORC_CUBIC : ORC_LINEAR, act);
    else
        run_level(B, l, interp, order, act);
}

static int block_run(block* B, const uint8_t* interp, const uint8_t* order, action* act)
{
    int l;
    for (l = B->G->L - 1; l >= 0; l--) {
        run_level_any(B, l, interp[l], order + 3 * l, act);
        if (act->status) return act->status;
    }
    if (!block_complete(B)) return ORC_EMISSED;
    return ORC_OK;
}

/* Write a finished block into the global arrays; a point written earlier
 * by another block must carry identical bits. */
static int block_store(const block* B, uint8_t* g_codes, float* g_rec, uint8_t* written)
{
    const geom* G = B->G;
    int c0, c1, c2;
    for (c0 = 0; c0 <= B->e[0]; c0++)
        for (c1 = 0; c1 <= B->e[1]; c1++)
            for (c2 = 0; c2 <= B->e[2]; c2++) {
                int li = lidx(B, c0, c1, c2);
                int64_t g = gindex(G, B->o[0] + c0, B->o[1] + c1, B->o[2] + c2);
                if (written[g]) {
                    if (g_codes && g_codes[g] != B->code[li]) return ORC_EFACE;
                    if (memcmp(&g_rec[g], &B->rec[li], sizeof(float)) != 0) return ORC_EFACE;
                } else {
                    if (g_codes) g_codes[g] = B->code[li];
                    g_rec[g] = B->rec[li];
                    written[g] = 1;
                }
            }
    return ORC_OK;
}

typedef struct {
    float* orig;
    float* rec;
    uint8_t* known;
    uint8_t* code;
} block_mem;

static int block_mem_alloc(block_mem* M, int A)
{
    size_t V = (size_t)(A + 1) * (A + 1) * (A + 1);
    M->orig = (float*)malloc(V * sizeof(float));
    M->rec = (float*)malloc(V * sizeof(float));
    M->known = (uint8_t*)malloc(V);
    M->code = (uint8_t*)malloc(V);
    if (!M->orig || !M->rec || !M->known || !M->code) return ORC_ENOMEM;
    return ORC_OK;
}

static void block_mem_free(block_mem* M)
{
    free(M->orig);
    free(M->rec);
    free(M->known);
    free(M->code);
}

static void block_attach(block* B, block_mem* M)
{
    B->orig = M->orig;
    B->rec = M->rec;
    B->known = M->known;
    B->code = M->code;
}

/* ------------------------------------------------------------------------ */
/* Compress.                                                                */
/*   consts = {eb_f, ebx2_f, r_f}.                                          */
/*   tiles / ntiles: optional list of linear block ids (row-major over the  */
/*   block grid); NULL = every block.  Only the listed blocks are written.  */
/*   Outputs (codes, recon: N entries; anchors: na0*na1*na2) are written    */
/*   only at points of processed blocks.                                    */
/* ------------------------------------------------------------------------ */
int hi_oracle_compress(const int64_t dims[3], int A, const uint8_t* interp, const uint8_t* order,
                       const float* consts, const float* x, const int64_t* tiles, int64_t ntiles,
                       uint8_t* codes, float* anchors, float* recon)
{
    geom G;
    block B;
    block_mem M;
    action act;
    uint8_t* written;
    int64_t k, nblocks;
    int rc = geom_init(&G, dims, A);
    if (rc) return rc;
    rc = check_levels(G.L, interp, order);
    if (rc) return rc;
    nblocks = G.nb[0] * G.nb[1] * G.nb[2];
    if (block_mem_alloc(&M, A)) {
        block_mem_free(&M);
        return ORC_ENOMEM;
    }
    written = (uint8_t*)calloc((size_t)G.N, 1);
    if (!written) {
        block_mem_free(&M);
        return ORC_ENOMEM;
    }
    block_attach(&B, &M);
    memset(&act, 0, sizeof act);
    act.mode = MODE_COMPRESS;
    act.eb_f = consts[0];
    act.ebx2_f = consts[1];
    act.r_f = consts[2];

    for (k = 0; k < (tiles ? ntiles : nblocks); k++) {
        int64_t t = tiles ? tiles[k] : k;
        int64_t t0, t1, t2;
        if (t < 0 || t >= nblocks) {
            rc = ORC_EINVAL;
            break;
        }
        t0 = t / (G.nb[1] * G.nb[2]);
        t1 = (t / G.nb[2]) % G.nb[1];
        t2 = t % G.nb[2];
        block_init(&B, &G, t0, t1, t2);
        block_seed(&B, x, NULL, MODE_COMPRESS);
        rc = block_run(&B, interp, order, &act);
        if (rc) break;
        rc = block_store(&B, codes, recon, written);
        if (rc) break;
    }
    if (!rc && anchors) {
        /* anchors of processed points, verbatim (Sec. 3.2) */
        int64_t a0, a1, a2;
        for (a0 = 0; a0 < G.na[0]; a0++)
            for (a1 = 0; a1 < G.na[1]; a1++)
                for (a2 = 0; a2 < G.na[2]; a2++) {
                    int64_t g = gindex(&G, a0 * A, a1 * A, a2 * A);
                    if (written[g]) anchors[(a0 * G.na[1] + a1) * G.na[2] + a2] = x[g];
                }
    }
    free(written);
    block_mem_free(&M);
    return rc;
}

/* Outliers and histogram from a complete code array: every non-anchor point
 * with code 0 is an outlier (index ascending, value = original); the
 * histogram counts the codes of the non-anchor points. */
int hi_oracle_collect(const int64_t dims[3], int A, const float* x, const uint8_t* codes,
                      uint32_t* out_idx, float* out_val, int64_t out_cap, int64_t* n_out, uint32_t* hist256)
{
    geom G;
    int64_t g0, g1, g2, cnt = 0;
    int rc = geom_init(&G, dims, A);
    if (rc) return rc;
    if (hist256) memset(hist256, 0, 256 * sizeof(uint32_t));
    for (g0 = 0; g0 < G.n[0]; g0++)
        for (g1 = 0; g1 < G.n[1]; g1++)
            for (g2 = 0; g2 < G.n[2]; g2++) {
                int64_t g = gindex(&G, g0, g1, g2);
                if (is_anchor(&G, g0, g1, g2)) continue;
                if (hist256) hist256[codes[g]]++;
                if (codes[g] == 0) {
                    if (cnt < out_cap) {
                        out_idx[cnt] = (uint32_t)g;
                        out_val[cnt] = x[g];
                    }
                    cnt++;
                }
            }
    *n_out = cnt;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Decompress: the same traversal; x' = p + (code-128)*fl(2 eps), or the    */
/* stored outlier value when the code is 0.                                 */
/* ------------------------------------------------------------------------ */
int hi_oracle_decompress(const int64_t dims[3], int A, const uint8_t* interp, const uint8_t* order,
                         float ebx2_f, const uint8_t* codes, const float* anchors, const uint32_t* out_idx,
                         const float* out_val, int64_t n_out, const int64_t* tiles, int64_t ntiles, float* recon)
{
    geom G;
    block B;
    block_mem M;
    action act;
    uint8_t *written, *outhas;
    float* outval;
    int64_t k, nblocks;
    int rc = geom_init(&G, dims, A);
    if (rc) return rc;
    rc = check_levels(G.L, interp, order);
    if (rc) return rc;
    nblocks = G.nb[0] * G.nb[1] * G.nb[2];
    if (block_mem_alloc(&M, A)) {
        block_mem_free(&M);
        return ORC_ENOMEM;
    }
    written = (uint8_t*)calloc((size_t)G.N, 1);
    outhas = (uint8_t*)calloc((size_t)G.N, 1);
    outval = (float*)calloc((size_t)G.N, sizeof(float));
    if (!written || !outhas || !outval) {
        rc = ORC_ENOMEM;
        goto done;
    }
    for (k = 0; k < n_out; k++) {
        if ((int64_t)out_idx[k] >= G.N) {
            rc = ORC_ECORRUPT;
            goto done;
        }
        outhas[out_idx[k]] = 1;
        outval[out_idx[k]] = out_val[k];
    }
    block_attach(&B, &M);
    memset(&act, 0, sizeof act);
    act.mode = MODE_DECOMPRESS;
    act.ebx2_f = ebx2_f;
    act.g_codes = codes;
    act.g_outval = outval;
    act.g_outhas = outhas;
    for (k = 0; k < (tiles ? ntiles : nblocks); k++) {
        int64_t t = tiles ? tiles[k] : k;
        int64_t t0, t1, t2;
        if (t < 0 || t >= nblocks) {
            rc = ORC_EINVAL;
            break;
        }
        t0 = t / (G.nb[1] * G.nb[2]);
        t1 = (t / G.nb[2]) % G.nb[1];
        t2 = t % G.nb[2];
        block_init(&B, &G, t0, t1, t2);
        block_seed(&B, NULL, anchors, MODE_DECOMPRESS);
        rc = block_run(&B, interp, order, &act);
        if (rc) break;
        rc = block_store(&B, NULL, recon, written);
        if (rc) break;
    }
done:
    free(written);
    free(outhas);
    free(outval);
    block_mem_free(&M);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Auto-tuning (Sec. 5.1.3).                                                */
/* ------------------------------------------------------------------------ */

/* Number of sampled blocks: 0.2 % of the points, in whole blocks. */
int64_t hi_oracle_tune_samples(const int64_t dims[3], int A)
{
    geom G;
    int64_t nblocks, vol = 1, m;
    int d;
    if (geom_init(&G, dims, A)) return -1;
    nblocks = G.nb[0] * G.nb[1] * G.nb[2];
    for (d = 0; d < 3; d++)
        if (G.n[d] > 1) vol *= A;
    m = (int64_t)floor(0.002 * (double)G.N / (double)vol + 0.5);
    if (m < 1) m = 1;
    if (m > nblocks) m = nblocks;
    return m;
}

/* Candidate configurations of one level, in enumeration order: the 1D
 * scheme, cubic before linear, within each the permutations of the active
 * dims in lexicographic order (inactive dims appended in ascending order);
 * then, when with_md is set and two or more dims are active, the
 * multi-dimensional scheme, cubic before linear (its order field is the
 * first permutation, unused).  Returns the count (at most 14). */
int hi_oracle_tune_configs(const int64_t dims[3], int with_md, uint8_t* interp_out, uint8_t* order_out)
{
    int act[3], na = 0, inact[3], ni = 0, d, i, cnt = 0, sp;
    int perms[6][3], np = 0;
    for (d = 0; d < 3; d++) {
        if (dims[d] > 1)
            act[na++] = d;
        else
            inact[ni++] = d;
    }
    if (na == 0) {
        perms[0][0] = 0;
        perms[0][1] = 1;
        perms[0][2] = 2;
        np = 1;
    } else if (na == 1) {
        perms[0][0] = act[0];
        np = 1;
    } else if (na == 2) {
        perms[0][0] = act[0];
        perms[0][1] = act[1];
        perms[1][0] = act[1];
        perms[1][1] = act[0];
        np = 2;
    } else {
        int a, b, c;
        for (a = 0; a < 3; a++)
            for (b = 0; b < 3; b++)
                for (c = 0; c < 3; c++)
                    if (a != b && b != c && a != c) {
                        perms[np][0] = a;
                        perms[np][1] = b;
                        perms[np][2] = c;
                        np++;
                    }
    }
    for (sp = 0; sp < 2; sp++) {
        for (i = 0; i < np; i++) {
            int q;
            interp_out[cnt] = (uint8_t)(sp == 0 ? ORC_CUBIC : ORC_LINEAR);
            if (na == 0) {
                for (q = 0; q < 3; q++) order_out[3 * cnt + q] = (uint8_t)perms[i][q];
            } else {
                for (q = 0; q < na; q++) order_out[3 * cnt + q] = (uint8_t)perms[i][q];
                for (q = 0; q < ni; q++) order_out[3 * cnt + na + q] = (uint8_t)inact[q];
            }
            cnt++;
        }
    }
    if (with_md && na >= 2) {
        for (sp = 0; sp < 2; sp++) {
            int q;
            interp_out[cnt] = (uint8_t)(sp == 0 ? ORC_MD_CUBIC : ORC_MD_LINEAR);
            for (q = 0; q < 3; q++) order_out[3 * cnt + q] = order_out[q];
            cnt++;
        }
    }
    return cnt;
}

/* err[l * ncfg + c]: sum over the sampled blocks of |x - p| for the points
 * of level l under configuration c, predictions from original values.
 * The sampled blocks are every (nblocks / m)-th block, starting at block 0. */
int hi_oracle_tune_errors(const int64_t dims[3], int A, int with_md, const float* x, double* err, int* ncfg_out)
{
    geom G;
    block B;
    block_mem M;
    action act;
    uint8_t cinterp[14], corder[42];
    uint8_t lvl_interp[ORC_MAX_LEVELS], lvl_order[3 * ORC_MAX_LEVELS];
    int64_t m, stride, k, nblocks;
    int ncfg, c, l, rc = geom_init(&G, dims, A);
    if (rc) return rc;
    nblocks = G.nb[0] * G.nb[1] * G.nb[2];
    m = hi_oracle_tune_samples(dims, A);
    stride = nblocks / m;
    ncfg = hi_oracle_tune_configs(dims, with_md, cinterp, corder);
    *ncfg_out = ncfg;
    for (k = 0; k < G.L * ncfg; k++) err[k] = 0.0;
    if (block_mem_alloc(&M, A)) {
        block_mem_free(&M);
        return ORC_ENOMEM;
    }
    block_attach(&B, &M);
    for (k = 0; k < m; k++) {
        int64_t t = k * stride;
        int64_t t0 = t / (G.nb[1] * G.nb[2]);
        int64_t t1 = (t / G.nb[2]) % G.nb[1];
        int64_t t2 = t % G.nb[2];
        for (l = G.L - 1; l >= 0; l--) {
            for (c = 0; c < ncfg; c++) {
                int ll, q;
                /* levels above l are irrelevant: open-loop predictions read
                 * originals; mark them known by running them with config c */
                for (ll = 0; ll < G.L; ll++) {
                    lvl_interp[ll] = cinterp[c];
                    for (q = 0; q < 3; q++) lvl_order[3 * ll + q] = corder[3 * c + q];
                }
                block_init(&B, &G, t0, t1, t2);
                block_seed(&B, x, NULL, MODE_TUNE);
                memset(&act, 0, sizeof act);
                act.mode = MODE_TUNE;
                for (ll = G.L - 1; ll > l; ll--) {
                    run_level_any(&B, ll, lvl_interp[ll], lvl_order + 3 * ll, &act);
                    if (act.status) break;
                }
                if (act.status) {
                    rc = act.status;
                    goto done;
                }
                act.err = 0.0;
                run_level_any(&B, l, cinterp[c], corder + 3 * c, &act);
                if (act.status) {
                    rc = act.status;
                    goto done;
                }
                err[l * ncfg + c] += act.err;
            }
        }
    }
done:
    block_mem_free(&M);
    return rc;
}

/* Per listed block (row-major block ids, in list order): err[(k * L + l) *
 * ncfg + c] = sum of |x - p| over the points of level l of block tiles[k]
 * under configuration c, predictions from original values -- the terms that
 * hi_oracle_tune_errors adds up over its sampled blocks.  Lets ranks that
 * hold parts of a field evaluate the global sample blocks they hold. */
int hi_oracle_tune_errors_tiles(const int64_t dims[3], int A, int with_md, const float* x, const int64_t* tiles,
                                int64_t ntiles, double* err, int* ncfg_out)
{
    geom G;
    block B;
    block_mem M;
    action act;
    uint8_t cinterp[14], corder[42];
    int64_t k, nblocks;
    int ncfg, c, l, rc = geom_init(&G, dims, A);
    if (rc) return rc;
    nblocks = G.nb[0] * G.nb[1] * G.nb[2];
    ncfg = hi_oracle_tune_configs(dims, with_md, cinterp, corder);
    *ncfg_out = ncfg;
    for (k = 0; k < ntiles * G.L * ncfg; k++) err[k] = 0.0;
    if (block_mem_alloc(&M, A)) {
        block_mem_free(&M);
        return ORC_ENOMEM;
    }
    block_attach(&B, &M);
    for (k = 0; k < ntiles; k++) {
        const int64_t t = tiles[k];
        int64_t t0, t1, t2;
        if (t < 0 || t >= nblocks) {
            rc = ORC_EINVAL;
            goto done;
        }
        t0 = t / (G.nb[1] * G.nb[2]);
        t1 = (t / G.nb[2]) % G.nb[1];
        t2 = t % G.nb[2];
        for (l = G.L - 1; l >= 0; l--) {
            for (c = 0; c < ncfg; c++) {
                int ll;
                block_init(&B, &G, t0, t1, t2);
                block_seed(&B, x, NULL, MODE_TUNE);
                memset(&act, 0, sizeof act);
                act.mode = MODE_TUNE;
                for (ll = G.L - 1; ll > l; ll--) {
                    run_level_any(&B, ll, cinterp[c], corder + 3 * c, &act);
                    if (act.status) break;
                }
                if (act.status) {
                    rc = act.status;
                    goto done;
                }
                act.err = 0.0;
                run_level_any(&B, l, cinterp[c], corder + 3 * c, &act);
                if (act.status) {
                    rc = act.status;
                    goto done;
                }
                err[(k * G.L + l) * ncfg + c] = act.err;
            }
        }
    }
done:
    block_mem_free(&M);
    return rc;
}

/* Per level, the configuration with the smallest error; ties go to the
 * first in enumeration order. */
int hi_oracle_tune_select(const int64_t dims[3], int A, int with_md, const double* err, uint8_t* interp, uint8_t* order)
{
    uint8_t cinterp[14], corder[42];
    int ncfg = hi_oracle_tune_configs(dims, with_md, cinterp, corder);
    int L = ilog2_exact(A), l, c, q;
    if (L < 1) return ORC_EINVAL;
    for (l = 0; l < L; l++) {
        int best = 0;
        for (c = 1; c < ncfg; c++)
            if (err[l * ncfg + c] < err[l * ncfg + best]) best = c;
        interp[l] = cinterp[best];
        for (q = 0; q < 3; q++) order[3 * l + q] = corder[3 * best + q];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Traversal trace: for every point, the level, the dimension and the       */
/* stencil case of its prediction (-1 for anchors).  Shared face points     */
/* must be traced identically by both blocks.                               */
/* ------------------------------------------------------------------------ */
int hi_oracle_trace(const int64_t dims[3], int A, const uint8_t* interp, const uint8_t* order, int8_t* lvl,
                    int8_t* dir, int8_t* kase)
{
    geom G;
    block B;
    block_mem M;
    action act;
    int64_t t, nblocks, g;
    float* zeros;
    int rc = geom_init(&G, dims, A);
    if (rc) return rc;
    rc = check_levels(G.L, interp, order);
    if (rc) return rc;
    nblocks = G.nb[0] * G.nb[1] * G.nb[2];
    zeros = (float*)calloc((size_t)G.N, sizeof(float));
    if (!zeros || block_mem_alloc(&M, A)) {
        free(zeros);
        return ORC_ENOMEM;
    }
    for (g = 0; g < G.N; g++) {
        lvl[g] = -1;
        dir[g] = -1;
        kase[g] = -1;
    }
    block_attach(&B, &M);
    memset(&act, 0, sizeof act);
    act.mode = MODE_TUNE;
    act.t_lvl = lvl;
    act.t_dir = dir;
    act.t_case = kase;
    for (t = 0; t < nblocks; t++) {
        block_init(&B, &G, t / (G.nb[1] * G.nb[2]), (t / G.nb[2]) % G.nb[1], t % G.nb[2]);
        block_seed(&B, zeros, NULL, MODE_TUNE);
        rc = block_run(&B, interp, order, &act);
        if (rc) break;
    }
    free(zeros);
    block_mem_free(&M);
    return rc;
}

/* ---------------------------------------------------------------------------
 * Quantization-code reordering (Sec. 5.2.2, Eq. 3).
 *
 * The code of the point (x, y, z) (x slowest; dims dx, dy, dz) goes to
 * position I(x, y, z) of a 1D sequence in which the codes of each
 * interpolation level lie together, coarser levels first.  The level of a
 * point is the largest l <= log2 A such that 2^l divides x, y and z;
 * prefix(l) = fx(l) fy(l) fz(l) is the number of points on coarser levels,
 * with f(0) = floor((d + 1) / 2) and f(k + 1) = floor((f(k) + 1) / 2), and
 * prefix(log2 A) = 0.
 *
 * Reading: Eq. 3 spells out the rank within a level for l = 0 on the global
 * grid -- the row-major index x dy dz + y dz + z minus the number of points
 * with three even coordinates that precede it.  For 0 < l < log2 A the same
 * rank is taken on the stride-2^l subgrid (coordinates x / 2^l, ..., whose
 * dims are f(l - 1)), which is the reading under which prefix(l) counts the
 * coarser points; the anchors (l = log2 A) come first, in the row-major
 * order of the anchor grid.
 *
 * I[p] for every point p in row-major order.
 * ------------------------------------------------------------------------- */
static int64_t half_up(int64_t d) { return (d + 1) / 2; }  /* floor((d + 1) / 2) */

int hi_oracle_reorder_index(const int64_t dims[3], int A, int64_t* I)
{
    const int L = ilog2_exact(A);
    if (L < 1 || L > 6) return 1;
    for (int d = 0; d < 3; ++d)
        if (dims[d] < 1) return 1;
    /* sub[l][d]: points per dim of the stride-2^l grid; sub[0] = dims, and
       sub[l + 1] = f(l) of Eq. 3 */
    int64_t sub[8][3];
    for (int d = 0; d < 3; ++d) {
        sub[0][d] = dims[d];
        for (int l = 0; l < L; ++l) sub[l + 1][d] = half_up(sub[l][d]);
    }
    int64_t prefix[8];
    for (int l = 0; l < L; ++l) prefix[l] = sub[l + 1][0] * sub[l + 1][1] * sub[l + 1][2];
    prefix[L] = 0;
    int64_t p = 0;
    for (int64_t x = 0; x < dims[0]; ++x)
        for (int64_t y = 0; y < dims[1]; ++y)
            for (int64_t z = 0; z < dims[2]; ++z, ++p) {
                int l = 0;
                while (l < L) {
                    const int64_t s = (int64_t)1 << (l + 1);
                    if (x % s != 0 || y % s != 0 || z % s != 0) break;
                    ++l;
                }
                const int64_t xs = x >> l, ys = y >> l, zs = z >> l;
                const int64_t Dy = sub[l][1], Dz = sub[l][2];
                int64_t rank = xs * Dy * Dz + ys * Dz + zs;
                if (l < L) {
                    rank -= half_up(xs) * half_up(Dy) * half_up(Dz);
                    if (xs % 2 == 0) rank -= half_up(ys) * half_up(Dz);
                    if (xs % 2 == 0 && ys % 2 == 0) rank -= half_up(zs);
                }
                I[p] = prefix[l] + rank;
            }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Throughput-mode lossless pipeline TCMS1-BIT1-RRE1 (Sec. 5.2.3) over a byte
 * sequence (the reordered codes).  The paper names the stages and what each
 * does; chunking, bit-plane order, recursion depth and the container are
 * not given, so this format is a reading:
 *
 *   stream   = u64 n | u32 chunk (16384) | u32 nchunks | u32 size[nchunks]
 *              | zero padding to 16 bytes | payloads, each padded to 16
 *   size[k]  = padded payload bytes; bit 31 set: the chunk is stored raw
 *   chunk k  = bytes [16384 k, min(16384 (k + 1), n)), m of them
 *   TCMS1    t = (b << 1) ^ (b >> 7) on the byte read as a signed int8
 *              (two's complement -> magnitude-sign; code 128 -> 0xff)
 *   BIT1     t zero-padded to m' = m rounded up to 64; plane p = 0..7 holds
 *              bit 7 - p of every element: byte j of a plane has element
 *              8 j + b at bit b; planes in order, m' / 8 bytes each
 *   RRE1     over a byte string v of length L: bitmap bit i = (v[i] !=
 *              v[i - 1]) with v[-1] = 0, byte j of the bitmap holding bits
 *              8 j .. 8 j + 7 (LSB first), ceil(L / 8) bytes; kept = the
 *              bytes whose bit is set, in order.  Levels: v_0 = the shuffled
 *              chunk, v_{r+1} = bitmap of v_r, until a level has L_R <= 64
 *              bytes, which is stored as is.
 *   payload  = v_R | kept_{R-1} | ... | kept_0 (decodable front to back);
 *              if that is longer than m the chunk is stored raw (m bytes).
 * ------------------------------------------------------------------------- */
#define TP_CHUNK 16384
#define TP_RAW 0x80000000u

static uint8_t tcms1(uint8_t b) { return (uint8_t)((b << 1) ^ ((b & 0x80) ? 0xff : 0x00)); }
static uint8_t tcms1_inv(uint8_t t) { return (uint8_t)((t >> 1) ^ ((t & 1) ? 0xff : 0x00)); }

/* RRE of v[0..L): bitmap into bm (ceil(L/8) bytes), kept bytes into kept; returns their count */
static int64_t rre_level(const uint8_t* v, int64_t L, uint8_t* bm, uint8_t* kept)
{
    int64_t nk = 0;
    memset(bm, 0, (size_t)((L + 7) / 8));
    for (int64_t i = 0; i < L; ++i) {
        const uint8_t prev = i ? v[i - 1] : 0;
        if (v[i] != prev) {
            bm[i / 8] |= (uint8_t)(1u << (i % 8));
            kept[nk++] = v[i];
        }
    }
    return nk;
}

static int64_t tp_chunk_encode(const uint8_t* s, int64_t m, uint8_t* out /* >= m + 64 */, int* raw)
{
    const int64_t mp = (m + 63) / 64 * 64;
    uint8_t* t = calloc((size_t)mp, 1);
    uint8_t* u = calloc((size_t)mp, 1);
    /* levels */
    uint8_t* lv[8];
    uint8_t* kept[8];
    int64_t L[8], nk[8];
    if (!t || !u) { free(t); free(u); return -1; }
    for (int64_t i = 0; i < m; ++i) t[i] = tcms1(s[i]);
    const int64_t pl = mp / 8;
    for (int p = 0; p < 8; ++p)
        for (int64_t e = 0; e < mp; ++e)
            if ((t[e] >> (7 - p)) & 1) u[p * pl + e / 8] |= (uint8_t)(1u << (e % 8));
    lv[0] = u;
    L[0] = mp;
    int R = 0;
    while (L[R] > 64) {
        lv[R + 1] = malloc((size_t)((L[R] + 7) / 8));
        kept[R] = malloc((size_t)L[R]);
        L[R + 1] = (L[R] + 7) / 8;
        nk[R] = rre_level(lv[R], L[R], lv[R + 1], kept[R]);
        ++R;
    }
    int64_t total = L[R];
    for (int r = 0; r < R; ++r) total += nk[r];
    int64_t len;
    if (total > m) {
        memcpy(out, s, (size_t)m);
        len = m;
        *raw = 1;
    } else {
        int64_t o = 0;
        memcpy(out + o, lv[R], (size_t)L[R]);
        o += L[R];
        for (int r = R - 1; r >= 0; --r) {
            memcpy(out + o, kept[r], (size_t)nk[r]);
            o += nk[r];
        }
        len = o;
        *raw = 0;
    }
    for (int r = 0; r < R; ++r) { free(lv[r + 1]); free(kept[r]); }
    free(t);
    free(u);
    return len;
}

static int64_t tp_header_bytes(int64_t nchunks) { return (16 + 4 * nchunks + 15) / 16 * 16; }

/* Upper bound of the stream size for n input bytes. */
int64_t hi_oracle_tp_bound(int64_t n)
{
    const int64_t nc = (n + TP_CHUNK - 1) / TP_CHUNK;
    return tp_header_bytes(nc) + nc * 16 + n + 15;
}

int hi_oracle_tp_encode(const uint8_t* in, int64_t n, uint8_t* out, int64_t cap, int64_t* out_len)
{
    if (n < 0 || (n && !in) || !out || !out_len) return 1;
    const int64_t nc = (n + TP_CHUNK - 1) / TP_CHUNK;
    if (cap < hi_oracle_tp_bound(n)) return 1;
    memset(out, 0, (size_t)tp_header_bytes(nc));
    memcpy(out, &n, 8);
    const uint32_t ch = TP_CHUNK, nc32 = (uint32_t)nc;
    memcpy(out + 8, &ch, 4);
    memcpy(out + 12, &nc32, 4);
    int64_t o = tp_header_bytes(nc);
    uint8_t* buf = malloc(TP_CHUNK + 64);
    if (!buf) return 2;
    for (int64_t k = 0; k < nc; ++k) {
        const int64_t m = (k + 1) * TP_CHUNK <= n ? TP_CHUNK : n - k * TP_CHUNK;
        int raw = 0;
        const int64_t len = tp_chunk_encode(in + k * TP_CHUNK, m, buf, &raw);
        if (len < 0) { free(buf); return 2; }
        const int64_t pad = (len + 15) / 16 * 16;
        memcpy(out + o, buf, (size_t)len);
        memset(out + o + len, 0, (size_t)(pad - len));
        const uint32_t sz = (uint32_t)pad | (raw ? TP_RAW : 0u);
        memcpy(out + 16 + 4 * k, &sz, 4);
        o += pad;
    }
    free(buf);
    *out_len = o;
    return 0;
}

int hi_oracle_tp_decode(const uint8_t* in, int64_t len, uint8_t* out, int64_t n)
{
    if (len < 16 || !in || (n && !out)) return 1;
    int64_t n_s;
    uint32_t ch, nc;
    memcpy(&n_s, in, 8);
    memcpy(&ch, in + 8, 4);
    memcpy(&nc, in + 12, 4);
    if (n_s != n || ch != TP_CHUNK || (int64_t)nc != (n + TP_CHUNK - 1) / TP_CHUNK) return 15;
    int64_t o = tp_header_bytes(nc);
    if (o > len) return 15;
    uint8_t* lv[9];
    for (int r = 0; r < 9; ++r) lv[r] = malloc(TP_CHUNK + 64);
    int rc = 0;
    for (int64_t k = 0; k < (int64_t)nc && rc == 0; ++k) {
        uint32_t sz;
        memcpy(&sz, in + 16 + 4 * k, 4);
        const int64_t pad = sz & ~TP_RAW;
        const int64_t m = (k + 1) * TP_CHUNK <= n ? TP_CHUNK : n - k * TP_CHUNK;
        if (o + pad > len) { rc = 15; break; }
        const uint8_t* p = in + o;
        if (sz & TP_RAW) {
            if (pad < m) { rc = 15; break; }
            memcpy(out + k * TP_CHUNK, p, (size_t)m);
        } else {
            const int64_t mp = (m + 63) / 64 * 64;
            int64_t L[9];
            L[0] = mp;
            int R = 0;
            while (L[R] > 64) { L[R + 1] = (L[R] + 7) / 8; ++R; }
            int64_t q = 0;
            if (L[R] > pad) { rc = 15; break; }
            memcpy(lv[R], p, (size_t)L[R]);
            q = L[R];
            for (int r = R - 1; r >= 0 && rc == 0; --r) {
                /* v_r from its bitmap v_{r+1} and the kept bytes */
                uint8_t prev = 0;
                for (int64_t i = 0; i < L[r]; ++i) {
                    if ((lv[r + 1][i / 8] >> (i % 8)) & 1) {
                        if (q >= pad) { rc = 15; break; }
                        prev = p[q++];
                    }
                    lv[r][i] = prev;
                }
            }
            if (rc) break;
            const int64_t pl = mp / 8;
            for (int64_t e = 0; e < m; ++e) {
                uint8_t t = 0;
                for (int pp = 0; pp < 8; ++pp)
                    t |= (uint8_t)(((lv[0][pp * pl + e / 8] >> (e % 8)) & 1) << (7 - pp));
                out[k * TP_CHUNK + e] = tcms1_inv(t);
            }
        }
        o += pad;
    }
    for (int r = 0; r < 9; ++r) free(lv[r]);
    return rc;
}

/* ---------------------------------------------------------------------------
 * Compression-ratio-mode lossless pipeline HF-RRE4-TCMS8-RZE1 (Sec. 5.2.3)
 * over a byte sequence (the reordered codes).  The paper names the stages:
 * Huffman coding, then repeat elimination on 4-byte symbols with a bitmap
 * compressed recursively, the magnitude-sign transform (w << 1) ^ (w >> 63)
 * on 8-byte words, and zero elimination on bytes "similar to RRE4".  The
 * code construction, block sizes and container are not given; readings:
 *
 *   HF       frequencies of the n symbols; Huffman code lengths from the
 *            tree that repeatedly merges the two lowest-ranked live nodes,
 *            nodes ranked by (weight, creation index) with the leaves
 *            created first in increasing symbol order and internal nodes
 *            numbered on from there as they are formed; a symbol's length
 *            is its leaf's depth (a lone symbol: 1).  While a length exceeds
 *            16, every nonzero weight w becomes max(1, w >> 1) and the tree
 *            is built again.  Canonical codes: symbols in (length, symbol)
 *            order, the first gets 0, each next (prev + 1) << (its length -
 *            the previous length).  Symbols are coded in blocks of 4096; a
 *            block's code bits go out most significant first (bit 7 of a
 *            byte first) and are padded with zero bits to a multiple of 32;
 *            the HF bytes are the blocks' padded bit strings in order.
 *   RRE4     on a chunk of m bytes (m a multiple of 4): word bitmap bit i =
 *            (word i != word i-1), word -1 = 0, LSB first; the bitmap is
 *            reduced by RRE1 levels (as in the throughput pipeline) until a
 *            level has at most 64 bytes; output = top level | kept bytes of
 *            the levels below, top down | kept words.
 *   TCMS8    every whole little-endian 8-byte word t of that output becomes
 *            (t << 1) ^ (t >> 63) (arithmetic shift), the tail bytes stay.
 *   RZE1     on the m1 bytes of that: levels v_0 = the bytes, v_{r+1} = the
 *            bitmap of (v_r[i] != 0), until a level has at most 64 bytes;
 *            payload = v_R | nonzero bytes of v_{R-1} | ... | of v_0.  A
 *            chunk whose payload is longer than m is stored raw.
 *   stream   u64 n | u32 4096 | u32 nblocks | u64 H (HF bytes) | u32 16384 |
 *            u32 nchunks | u8 length[256] | u32 words[nblocks] |
 *            u16 sub[3 nblocks] | zero padding to 4 |
 *            (u32 size, u32 m1)[nchunks] | zero padding to 16 | payloads,
 *            each padded to 16 (size = padded bytes, bit 31 = raw; m1 = the
 *            RRE4 output length, 0 for a raw chunk).  sub[3 b + j - 1]
 *            (j = 1, 2, 3) is the bit offset in block b of its symbol
 *            1024 j, or the block's bit count when it has fewer symbols:
 *            four independent starting points a block for a decoder.
 * ------------------------------------------------------------------------- */
#define HF_LMAX 16
#define HF_BLOCK 4096
#define CR_CHUNK 16384

/* Tree lengths for weights w (0 = absent); returns the longest length. */
static int hf_tree_lengths(const uint64_t* w, uint8_t* len)
{
    uint64_t wt[511];
    int parent[511], alive[511], sym[256];
    int k = 0, nodes, i, step;
    int maxlen = 0;
    memset(len, 0, 256);
    for (i = 0; i < 256; ++i)
        if (w[i] > 0) {
            wt[k] = w[i];
            sym[k] = i;
            alive[k] = 1;
            parent[k] = -1;
            ++k;
        }
    if (k == 0) return 0;
    if (k == 1) {
        len[sym[0]] = 1;
        return 1;
    }
    nodes = k;
    for (step = 0; step < k - 1; ++step) {
        int a = -1, b = -1;
        for (i = 0; i < nodes; ++i) { /* the two lowest (weight, index) live nodes */
            if (!alive[i]) continue;
            if (a < 0 || wt[i] < wt[a]) {
                b = a;
                a = i;
            } else if (b < 0 || wt[i] < wt[b]) {
                b = i;
            }
        }
        wt[nodes] = wt[a] + wt[b];
        alive[nodes] = 1;
        parent[nodes] = -1;
        parent[a] = nodes;
        parent[b] = nodes;
        alive[a] = 0;
        alive[b] = 0;
        ++nodes;
    }
    for (i = 0; i < k; ++i) {
        int d = 0, j = i;
        while (parent[j] >= 0) {
            j = parent[j];
            ++d;
        }
        len[sym[i]] = (uint8_t)d;
        if (d > maxlen) maxlen = d;
    }
    return maxlen;
}

/* Huffman code lengths (at most 16) of a 256-bin frequency table. */
int hi_oracle_hf_lengths(const uint64_t* freq, uint8_t* len)
{
    uint64_t w[256];
    int i;
    memcpy(w, freq, sizeof w);
    while (hf_tree_lengths(w, len) > HF_LMAX)
        for (i = 0; i < 256; ++i)
            if (w[i] > 0) w[i] = (w[i] >> 1) ? (w[i] >> 1) : 1;
    return 0;
}

/* Canonical codes from the lengths. */
static void hf_canonical(const uint8_t* len, uint32_t* code)
{
    int l, v, first = 1, pl = 0;
    uint32_t c = 0;
    memset(code, 0, 256 * sizeof(uint32_t));
    for (l = 1; l <= HF_LMAX; ++l)
        for (v = 0; v < 256; ++v)
            if (len[v] == l) {
                c = first ? 0u : ((c + 1u) << (l - pl));
                first = 0;
                pl = l;
                code[v] = c;
            }
}

/* Zero-elimination level: bitmap of (v[i] != 0) into bm, nonzero bytes into kept. */
static int64_t rze_level(const uint8_t* v, int64_t L, uint8_t* bm, uint8_t* kept)
{
    int64_t nk = 0;
    memset(bm, 0, (size_t)((L + 7) / 8));
    for (int64_t i = 0; i < L; ++i)
        if (v[i] != 0) {
            bm[i / 8] |= (uint8_t)(1u << (i % 8));
            kept[nk++] = v[i];
        }
    return nk;
}

/* Levels of a byte string (zero elimination or repeat elimination) until a
 * level has at most 64 bytes; writes v_R | kept_{R-1} | ... | kept_0 to out
 * and returns its length. */
static int64_t reduce_levels(const uint8_t* s, int64_t L0, int zero, uint8_t* out)
{
    const uint8_t* lv[16];
    uint8_t* own[16];
    uint8_t* kept[16];
    int64_t L[16], nk[16], o = 0;
    int R = 0, r;
    lv[0] = s;
    L[0] = L0;
    while (L[R] > 64) {
        own[R + 1] = malloc((size_t)((L[R] + 7) / 8));
        kept[R] = malloc((size_t)L[R]);
        L[R + 1] = (L[R] + 7) / 8;
        nk[R] = zero ? rze_level(lv[R], L[R], own[R + 1], kept[R]) : rre_level(lv[R], L[R], own[R + 1], kept[R]);
        lv[R + 1] = own[R + 1];
        ++R;
    }
    memcpy(out, lv[R], (size_t)L[R]);
    o = L[R];
    for (r = R - 1; r >= 0; --r) {
        memcpy(out + o, kept[r], (size_t)nk[r]);
        o += nk[r];
    }
    for (r = 0; r < R; ++r) {
        free(own[r + 1]);
        free(kept[r]);
    }
    return o;
}

/* Inverse of reduce_levels: rebuilds the L0 bytes of level 0 into dst from
 * p[0..avail); returns the bytes consumed or -1. */
static int64_t expand_levels(const uint8_t* p, int64_t avail, int64_t L0, int zero, uint8_t* dst)
{
    int64_t L[16], q;
    uint8_t* lv[16];
    int R = 0, r;
    L[0] = L0;
    while (L[R] > 64) {
        L[R + 1] = (L[R] + 7) / 8;
        ++R;
    }
    if (L[R] > avail) return -1;
    lv[0] = dst;
    for (r = 1; r <= R; ++r) lv[r] = malloc((size_t)L[r]);
    memcpy(lv[R], p, (size_t)L[R]);
    q = L[R];
    for (r = R - 1; r >= 0; --r) {
        uint8_t prev = 0;
        for (int64_t i = 0; i < L[r]; ++i) {
            if ((lv[r + 1][i / 8] >> (i % 8)) & 1) {
                if (q >= avail) {
                    q = -1;
                    break;
                }
                prev = p[q++];
                lv[r][i] = prev;
            } else {
                lv[r][i] = zero ? 0 : prev;
            }
        }
        if (q < 0) break;
    }
    for (r = 1; r <= R; ++r) free(lv[r]);
    return q;
}

static uint64_t ld64(const uint8_t* p)
{
    uint64_t v = 0;
    for (int b = 7; b >= 0; --b) v = (v << 8) | p[b];
    return v;
}

static void st64(uint8_t* p, uint64_t v)
{
    for (int b = 0; b < 8; ++b) p[b] = (uint8_t)(v >> (8 * b));
}

static uint64_t tcms8(uint64_t t) { return (t << 1) ^ ((t >> 63) ? ~(uint64_t)0 : 0); }
static uint64_t tcms8_inv(uint64_t u) { return (u >> 1) ^ ((u & 1) ? ~(uint64_t)0 : 0); }

/* One LC chunk: RRE4, TCMS8, RZE1.  out >= 2 m + 256; returns the payload length and m1. */
static int64_t cr_chunk_encode(const uint8_t* c, int64_t m, uint8_t* out, int64_t* m1_out, int* raw)
{
    const int64_t w = m / 4, L0 = (w + 7) / 8;
    uint8_t* bm = calloc((size_t)L0 + 1, 1);
    uint8_t* r = malloc((size_t)(2 * m + 256));
    int64_t nk = 0, m1, j, len;
    for (int64_t i = 0; i < w; ++i) {
        const int eq = i > 0 ? memcmp(c + 4 * i, c + 4 * (i - 1), 4) == 0
                             : (c[0] == 0 && c[1] == 0 && c[2] == 0 && c[3] == 0);
        if (!eq) {
            bm[i / 8] |= (uint8_t)(1u << (i % 8));
            ++nk;
        }
    }
    m1 = reduce_levels(bm, L0, 0, r);
    for (int64_t i = 0; i < w; ++i)
        if ((bm[i / 8] >> (i % 8)) & 1) {
            memcpy(r + m1, c + 4 * i, 4);
            m1 += 4;
        }
    for (j = 0; j + 8 <= m1; j += 8) st64(r + j, tcms8(ld64(r + j)));
    len = reduce_levels(r, m1, 1, out);
    if (len > m) {
        memcpy(out, c, (size_t)m);
        len = m;
        *raw = 1;
        m1 = 0;
    } else {
        *raw = 0;
    }
    *m1_out = m1;
    free(bm);
    free(r);
    (void)nk;
    return len;
}

#define HF_SUB 1024 /* symbols between the starting points of a block */
static int64_t cr_tab_off(int64_t nb) { return 288 + 4 * nb + (6 * nb + 3) / 4 * 4; }
static int64_t cr_header_bytes(int64_t nb, int64_t nc) { return (cr_tab_off(nb) + 8 * nc + 15) / 16 * 16; }

/* Upper bound of the stream size for n input bytes. */
int64_t hi_oracle_cr_bound(int64_t n)
{
    const int64_t nb = (n + HF_BLOCK - 1) / HF_BLOCK;
    const int64_t H = nb * HF_BLOCK * 2 + 4 * nb; /* at most 16 bits a symbol */
    const int64_t nc = (H + CR_CHUNK - 1) / CR_CHUNK;
    return cr_header_bytes(nb, nc) + H + 16 * nc + 16;
}

int hi_oracle_cr_encode(const uint8_t* in, int64_t n, uint8_t* out, int64_t cap, int64_t* out_len)
{
    uint64_t freq[256];
    uint8_t len[256];
    uint32_t code[256];
    int64_t nb, nc, H = 0, b, k, o;
    uint8_t *hf, *buf;
    uint32_t* words;
    uint16_t* sub;
    if (n < 0 || (n && !in) || !out || !out_len || cap < hi_oracle_cr_bound(n)) return 1;
    memset(freq, 0, sizeof freq);
    for (int64_t i = 0; i < n; ++i) freq[in[i]]++;
    hi_oracle_hf_lengths(freq, len);
    hf_canonical(len, code);
    nb = (n + HF_BLOCK - 1) / HF_BLOCK;
    hf = calloc((size_t)(nb * HF_BLOCK * 2 + 16), 1);
    words = calloc((size_t)nb + 1, sizeof(uint32_t));
    sub = calloc(3 * (size_t)nb + 2, sizeof(uint16_t));
    if (!hf || !words || !sub) {
        free(hf);
        free(words);
        free(sub);
        return 2;
    }
    for (b = 0; b < nb; ++b) { /* Huffman blocks, MSB first, padded to 32 bits */
        const int64_t s0 = b * HF_BLOCK, s1 = s0 + HF_BLOCK < n ? s0 + HF_BLOCK : n;
        int64_t p = 8 * H;
        for (int64_t i = s0; i < s1; ++i) {
            if (i > s0 && (i - s0) % HF_SUB == 0) sub[3 * b + (i - s0) / HF_SUB - 1] = (uint16_t)(p - 8 * H);
            const int l = len[in[i]];
            for (int t = l - 1; t >= 0; --t, ++p)
                if ((code[in[i]] >> t) & 1) hf[p / 8] |= (uint8_t)(0x80u >> (p % 8));
        }
        const int64_t bits = p - 8 * H;
        for (int j = 1; j <= 3; ++j)
            if (s0 + (int64_t)j * HF_SUB >= s1) sub[3 * b + j - 1] = (uint16_t)bits;
        words[b] = (uint32_t)((bits + 31) / 32);
        H += 4 * (int64_t)words[b];
    }
    nc = (H + CR_CHUNK - 1) / CR_CHUNK;
    memset(out, 0, (size_t)cr_header_bytes(nb, nc));
    memcpy(out, &n, 8);
    {
        const uint32_t hb = HF_BLOCK, nb32 = (uint32_t)nb, cc = CR_CHUNK, nc32 = (uint32_t)nc;
        memcpy(out + 8, &hb, 4);
        memcpy(out + 12, &nb32, 4);
        memcpy(out + 16, &H, 8);
        memcpy(out + 24, &cc, 4);
        memcpy(out + 28, &nc32, 4);
    }
    memcpy(out + 32, len, 256);
    memcpy(out + 288, words, 4 * (size_t)nb);
    memcpy(out + 288 + 4 * nb, sub, 6 * (size_t)nb);
    o = cr_header_bytes(nb, nc);
    buf = malloc(2 * CR_CHUNK + 256);
    for (k = 0; k < nc; ++k) {
        const int64_t m = (k + 1) * CR_CHUNK <= H ? CR_CHUNK : H - k * CR_CHUNK;
        int64_t m1 = 0;
        int raw = 0;
        const int64_t l = cr_chunk_encode(hf + k * CR_CHUNK, m, buf, &m1, &raw);
        const int64_t pad = (l + 15) / 16 * 16;
        const uint32_t sz = (uint32_t)pad | (raw ? TP_RAW : 0u), m1_32 = (uint32_t)m1;
        if (o + pad > cap) {
            free(buf);
            free(hf);
            free(words);
            free(sub);
            return 1;
        }
        memcpy(out + o, buf, (size_t)l);
        memset(out + o + l, 0, (size_t)(pad - l));
        memcpy(out + cr_tab_off(nb) + 8 * k, &sz, 4);
        memcpy(out + cr_tab_off(nb) + 8 * k + 4, &m1_32, 4);
        o += pad;
    }
    free(buf);
    free(hf);
    free(words);
    free(sub);
    *out_len = o;
    return 0;
}

int hi_oracle_cr_decode(const uint8_t* in, int64_t len_in, uint8_t* out, int64_t n)
{
    int64_t n_s, H, nb, nc, o, k, b, pos = 0;
    uint32_t hb, nb32, cc, nc32;
    uint8_t len[256], sorted[256];
    uint32_t code[256], cnt[HF_LMAX + 1], first[HF_LMAX + 1], offs[HF_LMAX + 1];
    uint8_t *hf, *r;
    int rc = 0;
    if (len_in < 288 || !in || (n && !out)) return 1;
    memcpy(&n_s, in, 8);
    memcpy(&hb, in + 8, 4);
    memcpy(&nb32, in + 12, 4);
    memcpy(&H, in + 16, 8);
    memcpy(&cc, in + 24, 4);
    memcpy(&nc32, in + 28, 4);
    nb = nb32;
    nc = nc32;
    if (n_s != n || hb != HF_BLOCK || cc != CR_CHUNK || nb != (n + HF_BLOCK - 1) / HF_BLOCK || H < 0 ||
        H > nb * HF_BLOCK * 2 + 4 * nb || nc != (H + CR_CHUNK - 1) / CR_CHUNK)
        return 15;
    o = cr_header_bytes(nb, nc);
    if (o > len_in) return 15;
    memcpy(len, in + 32, 256);
    for (int v = 0; v < 256; ++v)
        if (len[v] > HF_LMAX) return 15;
    hf_canonical(len, code);
    {   /* per length: how many symbols, the first code, where they start in (length, symbol) order */
        int nsorted = 0;
        for (int l = 1; l <= HF_LMAX; ++l) {
            cnt[l] = 0;
            offs[l] = (uint32_t)nsorted;
            first[l] = 0;
            for (int v = 0; v < 256; ++v)
                if (len[v] == l) {
                    if (cnt[l] == 0) first[l] = code[v];
                    sorted[nsorted++] = (uint8_t)v;
                    cnt[l]++;
                }
        }
    }
    hf = calloc((size_t)H + 16, 1);
    r = malloc(2 * CR_CHUNK + 256);
    for (k = 0; k < nc && !rc; ++k) { /* LC chunks back to HF bytes */
        uint32_t sz, m1;
        const int64_t m = (k + 1) * CR_CHUNK <= H ? CR_CHUNK : H - k * CR_CHUNK;
        memcpy(&sz, in + cr_tab_off(nb) + 8 * k, 4);
        memcpy(&m1, in + cr_tab_off(nb) + 8 * k + 4, 4);
        const int64_t pad = sz & ~TP_RAW;
        if (o + pad > len_in) {
            rc = 15;
            break;
        }
        if (sz & TP_RAW) {
            if (pad < m) rc = 15;
            else memcpy(hf + k * CR_CHUNK, in + o, (size_t)m);
        } else {
            const int64_t w = m / 4, L0 = (w + 7) / 8;
            int64_t q, j;
            if ((int64_t)m1 > 2 * CR_CHUNK + 128 || expand_levels(in + o, pad, m1, 1, r) < 0) {
                rc = 15;
                break;
            }
            for (j = 0; j + 8 <= (int64_t)m1; j += 8) st64(r + j, tcms8_inv(ld64(r + j)));
            {
                uint8_t* bm = malloc((size_t)L0 + 1);
                q = expand_levels(r, m1, L0, 0, bm);
                if (q < 0) rc = 15;
                uint8_t prev[4] = {0, 0, 0, 0};
                for (int64_t i = 0; i < w && !rc; ++i) {
                    if ((bm[i / 8] >> (i % 8)) & 1) {
                        if (q + 4 > (int64_t)m1) {
                            rc = 15;
                            break;
                        }
                        memcpy(prev, r + q, 4);
                        q += 4;
                    }
                    memcpy(hf + k * CR_CHUNK + 4 * i, prev, 4);
                }
                free(bm);
            }
        }
        o += pad;
    }
    /* Huffman blocks back to symbols (canonical decoding bit by bit) */
    for (b = 0; b < nb && !rc; ++b) {
        uint32_t words;
        const int64_t s0 = b * HF_BLOCK, s1 = s0 + HF_BLOCK < n ? s0 + HF_BLOCK : n;
        int64_t p = 8 * pos;
        memcpy(&words, in + 288 + 4 * b, 4);
        if (pos + 4 * (int64_t)words > H) {
            rc = 15;
            break;
        }
        for (int64_t i = s0; i < s1 && !rc; ++i) {
            uint32_t c = 0;
            int l, found = 0;
            if (i > s0 && (i - s0) % HF_SUB == 0) { /* a starting point: the table must agree */
                uint16_t so;
                memcpy(&so, in + 288 + 4 * nb + 2 * (3 * b + (i - s0) / HF_SUB - 1), 2);
                if ((int64_t)so != p - 8 * pos) {
                    rc = 15;
                    break;
                }
            }
            for (l = 1; l <= HF_LMAX && !found; ++l) {
                if (p >= 8 * (pos + 4 * (int64_t)words)) {
                    rc = 15;
                    break;
                }
                c = (c << 1) | (uint32_t)((hf[p / 8] >> (7 - p % 8)) & 1);
                ++p;
                /* canonical codes of length l are first[l] .. first[l] + count[l] - 1 */
                if (cnt[l] > 0 && c >= first[l] && c - first[l] < cnt[l]) {
                    out[i] = sorted[offs[l] + (c - first[l])];
                    found = 1;
                }
            }
            if (!found && !rc) rc = 15;
        }
        for (int j = 1; j <= 3 && !rc; ++j) { /* starting points past the block's end hold its bit count */
            uint16_t so;
            memcpy(&so, in + 288 + 4 * nb + 2 * (3 * b + j - 1), 2);
            if (s0 + (int64_t)j * HF_SUB >= s1 && (int64_t)so != p - 8 * pos) rc = 15;
        }
        pos += 4 * (int64_t)words;
    }
    free(hf);
    free(r);
    return rc;
}
