/*
 * hasf_oracle.c -- CPU oracle for the homotopic alternating sequential filter
 * (HASF) of Mahmoudi & Akil, "Real Time Topological Image Smoothing On Shared
 * Memory Parallel Machines" (arXiv:1603.09337).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded
 * restatement of what the method computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  The CUDA library
 * never links, loads or calls it, and the two share no code, header, table or
 * constant generator.  Every function below cites the passage of the paper it
 * follows; the readings taken where the paper is garbled or silent are stated
 * next to the code that takes them.
 *
 * Conventions
 *  - An image is w x h bytes, row-major: pixel (x, y) lives at [y*w + x],
 *    x grows to the right, y grows downward.  Non-zero means "object".
 *  - The box [0,w) x [0,h) is the only region that can change.  Every point of
 *    Z^2 outside it is background, fixed forever (Sec. 2 takes X to be a finite
 *    subset of the plane, so its complement contains the whole outside).
 *  - Distances are squared Euclidean distances, exact 64-bit integers
 *    (Sec. 2, distance d; the minus sign printed inside the root is read as a
 *    plus, the Euclidean norm the text names).
 *  - Adjacency pair (n, nbar) is (8,4) or (4,8) (Sec. 2); "conn" is n.
 *
 * Parity status: every function is pinned by the CPU tests (brute force,
 * global topology, closed forms, invariants, hand-worked examples).  The
 * composition of the whole filter (radii ascending, cutting before filling)
 * is pinned by the classical alternating sequential filter by disc unions,
 * which it equals on simply connected shapes, and by a hand-worked HASF_1
 * example on which the two orders of HC_1 and HF_1 differ.  The paper prints
 * no result of the filter on its own images, so no comparison with those
 * exists.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_INF (INT64_C(1) << 62)

/* ------------------------------------------------------------------------ */
/* Neighbourhood and simple points (Sec. 2, Gamma_4 / Gamma_8, T and Tbar).  */
/* ------------------------------------------------------------------------ */

/* The eight neighbours of a point, in the order used for neighbour codes:
 * bit k of a code is neighbour k.  E, NE, N, NW, W, SW, S, SE. */
static const int NB_DX[8] = {1, 1, 0, -1, -1, -1, 0, 1};
static const int NB_DY[8] = {0, -1, -1, -1, 0, 1, 1, 1};

/* n-adjacency between two distinct points (Sec. 2). */
static int adjacent(int n, int ax, int ay, int bx, int by)
{
    int dx = abs(ax - bx), dy = abs(ay - by);
    if (dx == 0 && dy == 0) return 0;
    if (n == 8) return dx <= 1 && dy <= 1;
    return dx + dy == 1;
}

/* Number of n-connected components of the neighbour subset `members` (bit k
 * set = neighbour k belongs to the subset) that contain a point n-adjacent to
 * the centre (0,0).  Plain flood fill over the eight positions.  This is
 * #C_n[x, Gamma_8^*(x) cap S] of Sec. 2. */
static int count_adjacent_components(int n, unsigned members)
{
    int label[8];
    for (int k = 0; k < 8; ++k) label[k] = -1;
    int ncomp = 0, counted = 0;
    for (int k = 0; k < 8; ++k) {
        if (!((members >> k) & 1u) || label[k] >= 0) continue;
        int stack[8], sp = 0;
        stack[sp++] = k;
        label[k] = ncomp;
        int touches_centre = 0;
        while (sp) {
            int a = stack[--sp];
            if (adjacent(n, NB_DX[a], NB_DY[a], 0, 0)) touches_centre = 1;
            for (int b = 0; b < 8; ++b) {
                if (((members >> b) & 1u) && label[b] < 0 &&
                    adjacent(n, NB_DX[a], NB_DY[a], NB_DX[b], NB_DY[b])) {
                    label[b] = ncomp;
                    stack[sp++] = b;
                }
            }
        }
        counted += touches_centre;
        ++ncomp;
    }
    return counted;
}

/* lut[code] = 1 iff a point whose neighbours form `code` is simple:
 * T(x, X) = 1 and Tbar(x, X) = 1 (the local characterisation of Sec. 2).
 * T counts n-components of the object neighbours, Tbar counts
 * nbar-components of the background neighbours, each restricted to those
 * adjacent to the centre.  Simplicity depends only on Gamma_8^*(x) cap X,
 * so the same table answers "may x be removed from X" (x in X) and "may x be
 * added to X" (x not in X).  Returns 0, or -1 for a bad conn. */
int hasf_oracle_simple_lut(int conn, uint8_t *lut)
{
    if (conn != 8 && conn != 4) return -1;
    int nbar = conn == 8 ? 4 : 8;
    for (unsigned code = 0; code < 256; ++code) {
        int t = count_adjacent_components(conn, code);
        int tbar = count_adjacent_components(nbar, (~code) & 0xFFu);
        lut[code] = (uint8_t)(t == 1 && tbar == 1);
    }
    return 0;
}

/* Neighbour code of (x, y) in image S; points outside the box read as 0. */
static unsigned neighbour_code(const uint8_t *S, int w, int h, int x, int y)
{
    unsigned code = 0;
    for (int k = 0; k < 8; ++k) {
        int nx = x + NB_DX[k], ny = y + NB_DY[k];
        if (nx >= 0 && nx < w && ny >= 0 && ny < h && S[(size_t)ny * w + nx])
            code |= 1u << k;
    }
    return code;
}

/* ------------------------------------------------------------------------ */
/* Exact squared Euclidean distance transform (Sec. 4.1, Meijster).          */
/* ------------------------------------------------------------------------ */

static int64_t floor_div(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) --q;
    return q;
}

/* Core two-phase transform on a grid with no outside:
 * d[p] = min over feature q of |p - q|^2, or ORACLE_INF without features.
 *
 * Phase 1 (Sec. 4.1, Algorithm 1): for every column, the vertical distance
 * g to the nearest feature pixel of that column, by a downward scan
 * (g = 0 on a feature, else the value above plus one) and an upward scan
 * (take the value below plus one when that is smaller).  "No feature in the
 * column" is the value w + h, larger than any real distance in the grid.
 *
 * Phase 2 (Sec. 4.1, Algorithm 2): for every row, d(x) = min_i (x-i)^2 + g(i)^2
 * is the lower envelope of the parabolas i -> (x-i)^2 + g(i)^2.  A left-to-
 * right scan keeps the parabolas that are part of the envelope (their apex
 * column and the first column where each starts to win); a right-to-left scan
 * reads the envelope back out.  Readings: the loop that discards parabolas
 * walks the stack DOWN (the listing prints an increment), and the separator
 * divides by 2(u - i) with floor division (the listing prints 2(u - 1)). */
static int edt_grid(const uint8_t *feat, int w, int h, int64_t *d)
{
    const int64_t none = (int64_t)w + (int64_t)h;
    int64_t *g = (int64_t *)malloc((size_t)w * h * sizeof(int64_t));
    int *apex = (int *)malloc((size_t)(w > 0 ? w : 1) * sizeof(int));
    int64_t *start = (int64_t *)malloc((size_t)(w > 0 ? w : 1) * sizeof(int64_t));
    if (!g || !apex || !start) { free(g); free(apex); free(start); return -1; }

    /* Phase 1: columns. */
    for (int x = 0; x < w; ++x) {
        g[x] = feat[x] ? 0 : none;
        for (int y = 1; y < h; ++y) {
            size_t p = (size_t)y * w + x;
            g[p] = feat[p] ? 0 : g[p - w] + 1;
        }
        for (int y = h - 2; y >= 0; --y) {
            size_t p = (size_t)y * w + x;
            if (g[p + w] < g[p]) g[p] = g[p + w] + 1;
        }
    }

    /* Phase 2: rows. */
    for (int y = 0; y < h; ++y) {
        const int64_t *gr = g + (size_t)y * w;
        int64_t *dr = d + (size_t)y * w;
#define PARAB(x, i) ((int64_t)((x) - (i)) * ((x) - (i)) + gr[i] * gr[i])
        int top = 0;
        apex[0] = 0;
        start[0] = 0;
        for (int u = 1; u < w; ++u) {
            while (top >= 0 && PARAB(start[top], apex[top]) > PARAB(start[top], u))
                --top;
            if (top < 0) {
                top = 0;
                apex[0] = u;
                start[0] = 0;
            } else {
                int i = apex[top];
                int64_t num = (int64_t)u * u - (int64_t)i * i + gr[u] * gr[u] - gr[i] * gr[i];
                int64_t first_win = 1 + floor_div(num, 2 * (int64_t)(u - i));
                if (first_win < w) {
                    ++top;
                    apex[top] = u;
                    start[top] = first_win;
                }
            }
        }
        for (int u = w - 1; u >= 0; --u) {
            dr[u] = PARAB(u, apex[top]);
            if (u == start[top]) --top;
        }
#undef PARAB
    }

    for (size_t p = 0; p < (size_t)w * h; ++p)
        if (d[p] >= none * none) d[p] = ORACLE_INF;
    free(g);
    free(apex);
    free(start);
    return 0;
}

/* Squared distance from every box point to the nearest point of the feature
 * set F.  F is `feat` inside the box; when outside_is_feature is non-zero, F
 * also contains every point outside the box (used for distances to the
 * complement of an object, whose complement contains the outside).  The outside
 * is represented by a one-pixel frame: the nearest outside point of any box
 * point lies orthogonally just across the nearest edge, so the frame gives
 * the same distances as the infinite outside. */
int hasf_oracle_edt(const uint8_t *feat, int w, int h, int outside_is_feature, int64_t *d)
{
    if (w < 1 || h < 1) return -1;
    if (!outside_is_feature) return edt_grid(feat, w, h, d);
    int W = w + 2, H = h + 2;
    uint8_t *f = (uint8_t *)malloc((size_t)W * H);
    int64_t *dd = (int64_t *)malloc((size_t)W * H * sizeof(int64_t));
    if (!f || !dd) { free(f); free(dd); return -1; }
    memset(f, 1, (size_t)W * H);
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x)
            f[(size_t)(y + 1) * W + x + 1] = feat[(size_t)y * w + x] ? 1 : 0;
    int rc = edt_grid(f, W, H, dd);
    if (rc == 0)
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x)
                d[(size_t)y * w + x] = dd[(size_t)(y + 1) * W + x + 1];
    free(f);
    free(dd);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Erosion and dilation by the Euclidean ball B_r (Sec. 2).                  */
/* ------------------------------------------------------------------------ */

/* delta_r(S) = union of B_r(x), x in S, restricted to the box:
 * the box points at squared distance <= r^2 from S. */
int hasf_oracle_dilate(const uint8_t *S, int w, int h, int r, uint8_t *out)
{
    int64_t *d = (int64_t *)malloc((size_t)w * h * sizeof(int64_t));
    if (!d) return -1;
    int rc = hasf_oracle_edt(S, w, h, 0, d);
    for (size_t p = 0; rc == 0 && p < (size_t)w * h; ++p)
        out[p] = d[p] <= (int64_t)r * r;
    free(d);
    return rc;
}

/* eps_r(S), dual of the dilation: the points whose whole ball B_r lies in S,
 * i.e. the points at squared distance > r^2 from the complement of S (which
 * contains the outside of the box). */
int hasf_oracle_erode(const uint8_t *S, int w, int h, int r, uint8_t *out)
{
    size_t n = (size_t)w * h;
    uint8_t *comp = (uint8_t *)calloc(n, 1);
    int64_t *d = (int64_t *)malloc(n * sizeof(int64_t));
    if (!comp || !d) { free(comp); free(d); return -1; }
    for (size_t p = 0; p < n; ++p) comp[p] = !S[p];
    int rc = hasf_oracle_edt(comp, w, h, 1, d);
    for (size_t p = 0; rc == 0 && p < n; ++p)
        out[p] = S[p] && d[p] > (int64_t)r * r;
    free(comp);
    free(d);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Constrained thinning H(Z, W) and thickening *H(Y, V) (Sec. 2, Sec. 4.2).  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t levels;   /* priority levels visited                        */
    int64_t rounds;   /* rounds (4 subfield passes each), all levels     */
    int64_t changes;  /* points removed or added                         */
    int64_t max_rounds_per_level;
} hasf_oracle_stats;

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Shared driver of H and *H.  `S` is the set being thinned (remove = 1) or
 * thickened (remove = 0); `K` is the constraint: for thinning the points that
 * must stay (W), for thickening the points that may be added (V).  A point p
 * is a candidate when it can change (p in S minus W, or p in V minus S) and its
 * priority prio[p] is <= the current level.
 *
 * Order (the paper fixes the priority -- increasing distance, Sec. 2 -- and
 * leaves ties open; this is the reading taken):
 *   for each level l, in increasing order of the distinct candidate
 *   priorities:
 *     repeat rounds until a whole round changes nothing; a round visits the
 *     four subfields (x mod 2, y mod 2) = (0,0), (1,0), (0,1), (1,1) in that
 *     order, each in raster order, and changes every candidate that is simple
 *     in the current set at the moment it is visited.
 * Two points of one subfield are never 8-adjacent, so changing one never
 * alters the neighbourhood of another point of the same subfield: within a
 * subfield, any visiting order gives the same result.  Rounds repeat until
 * stability, as the worklist of Sec. 4.2 (Algorithm 3) does.  The loop ends
 * because every round but the last changes at least one point and a point
 * changes at most once. */
static int homotopic_sweep(uint8_t *S, const uint8_t *K, const int64_t *prio,
                           int w, int h, int conn, int remove,
                           hasf_oracle_stats *st)
{
    uint8_t lut[256];
    if (hasf_oracle_simple_lut(conn, lut) != 0) return -1;
    size_t n = (size_t)w * h;

    int64_t *lv = (int64_t *)malloc((n ? n : 1) * sizeof(int64_t));
    if (!lv) return -1;
    size_t nl = 0;
    for (size_t p = 0; p < n; ++p) {
        int cand = remove ? (S[p] && !K[p]) : (!S[p] && K[p]);
        if (cand) lv[nl++] = prio[p];
    }
    qsort(lv, nl, sizeof(int64_t), cmp_i64);
    size_t nd = 0;
    for (size_t i = 0; i < nl; ++i)
        if (nd == 0 || lv[nd - 1] != lv[i]) lv[nd++] = lv[i];

    for (size_t li = 0; li < nd; ++li) {
        int64_t level = lv[li];
        int64_t rounds_here = 0;
        for (;;) {
            int64_t changed = 0;
            for (int s = 0; s < 4; ++s) {
                int sx = s & 1, sy = s >> 1;
                for (int y = sy; y < h; y += 2) {
                    for (int x = sx; x < w; x += 2) {
                        size_t p = (size_t)y * w + x;
                        int cand = remove ? (S[p] && !K[p]) : (!S[p] && K[p]);
                        if (!cand || prio[p] > level) continue;
                        if (lut[neighbour_code(S, w, h, x, y)]) {
                            S[p] = (uint8_t)!remove;
                            ++changed;
                        }
                    }
                }
            }
            ++rounds_here;
            if (st) st->changes += changed;
            if (!changed) break;
        }
        if (st) {
            st->levels += 1;
            st->rounds += rounds_here;
            if (rounds_here > st->max_rounds_per_level) st->max_rounds_per_level = rounds_here;
        }
    }
    free(lv);
    return 0;
}

/* H(Z, W): homotopic thinning of Z constrained by W -- simple points of
 * Z \ W removed in increasing order of prio (Sec. 2: ultimate constrained
 * skeleton, points taken by increasing distance to the background given by a
 * distance map computed beforehand).  Z is updated in place. */
int hasf_oracle_thin(uint8_t *Z, const uint8_t *W, const int64_t *prio, int w, int h,
                     int conn, hasf_oracle_stats *st)
{
    return homotopic_sweep(Z, W, prio, w, h, conn, 1, st);
}

/* *H(Y, V): homotopic thickening of Y constrained by V -- points of V \ Y that
 * are simple (for the complement of Y) are added, in increasing order of prio,
 * until stability (Sec. 2).  Y is updated in place. */
int hasf_oracle_thicken(uint8_t *Y, const uint8_t *V, const int64_t *prio, int w, int h,
                        int conn, hasf_oracle_stats *st)
{
    return homotopic_sweep(Y, V, prio, w, h, conn, 0, st);
}

/* ------------------------------------------------------------------------ */
/* Homotopic cutting, filling and the alternating sequential filter.        */
/* ------------------------------------------------------------------------ */

/* HC_r^C(X) = *H(Y, V), Y = H(X, eps_r(X) cup C), V = delta_r(Y) cap X
 * (Sec. 2, eq. (i)).  The thinning priority is the distance of each point of
 * X to the complement of X; the thickening priority is the distance to Y.
 * X is updated in place; C may be NULL (empty). */
int hasf_oracle_hc(uint8_t *X, const uint8_t *C, int w, int h, int r, int conn,
                   hasf_oracle_stats *st)
{
    size_t n = (size_t)w * h;
    int64_t r2 = (int64_t)r * r;
    uint8_t *comp = (uint8_t *)calloc(n, 1), *K = (uint8_t *)calloc(n, 1);
    int64_t *d = (int64_t *)malloc(n * sizeof(int64_t));
    int rc = -1;
    if (!comp || !K || !d) goto out;

    /* Y = H(X, eps_r(X) cup C), priority = distance to the complement of X. */
    for (size_t p = 0; p < n; ++p) comp[p] = !X[p];
    if (hasf_oracle_edt(comp, w, h, 1, d)) goto out;
    for (size_t p = 0; p < n; ++p)
        K[p] = (X[p] && d[p] > r2) || (C && C[p] && X[p]);
    if (hasf_oracle_thin(X, K, d, w, h, conn, st)) goto out;   /* X now holds Y */

    /* V = delta_r(Y) cap X_input; priority = distance to Y. */
    if (hasf_oracle_edt(X, w, h, 0, d)) goto out;
    for (size_t p = 0; p < n; ++p) K[p] = d[p] <= r2 && !comp[p];
    rc = hasf_oracle_thicken(X, K, d, w, h, conn, st);
out:
    free(comp);
    free(K);
    free(d);
    return rc;
}

/* HF_r^D(X) = H(Z, W), Z = *H(X, delta_r(X) cap complement(D)),
 * W = eps_r(Z) cup X (Sec. 2, eq. (ii)).  Reading: the printed W uses
 * eps_n(Y), but Y is not defined in (ii); by duality with (i) -- filling X is
 * cutting its complement -- the eroded set is Z.  The thickening priority is
 * the distance to X; the thinning priority is the distance to the complement
 * of Z.  X is updated in place; D may be NULL (empty). */
int hasf_oracle_hf(uint8_t *X, const uint8_t *D, int w, int h, int r, int conn,
                   hasf_oracle_stats *st)
{
    size_t n = (size_t)w * h;
    int64_t r2 = (int64_t)r * r;
    uint8_t *orig = (uint8_t *)malloc(n), *K = (uint8_t *)malloc(n);
    int64_t *d = (int64_t *)malloc(n * sizeof(int64_t));
    int rc = -1;
    if (!orig || !K || !d) goto out;
    memcpy(orig, X, n);

    /* Z = *H(X, delta_r(X) cap complement(D)), priority = distance to X. */
    if (hasf_oracle_edt(X, w, h, 0, d)) goto out;
    for (size_t p = 0; p < n; ++p) K[p] = d[p] <= r2 && !(D && D[p]);
    if (hasf_oracle_thicken(X, K, d, w, h, conn, st)) goto out;  /* X now holds Z */

    /* W = eps_r(Z) cup X_input, priority = distance to the complement of Z. */
    for (size_t p = 0; p < n; ++p) K[p] = !X[p];
    if (hasf_oracle_edt(K, w, h, 1, d)) goto out;
    for (size_t p = 0; p < n; ++p) K[p] = (X[p] && d[p] > r2) || orig[p];
    rc = hasf_oracle_thin(X, K, d, w, h, conn, st);
out:
    free(orig);
    free(K);
    free(d);
    return rc;
}

/* HASF_n^{C,D} = HF_n^D o HC_n^C o ... o HF_1^D o HC_1^C (Sec. 2): for
 * r = 1..rmax, a homotopic cutting then a homotopic filling by B_r.
 * in: w x h bytes, non-zero = object.  C (kept points) is taken as C cap X,
 * D (points never added) as D minus X, since Sec. 2 requires C within X and D
 * within its complement; either may be NULL.  out receives 0/1 bytes and may
 * alias in.  Returns 0, or -1 on bad arguments / allocation failure. */
int hasf_oracle_hasf(const uint8_t *in, const uint8_t *C, const uint8_t *D, int w, int h,
                     int rmax, int conn, uint8_t *out, hasf_oracle_stats *st)
{
    if (w < 1 || h < 1 || rmax < 0 || (conn != 8 && conn != 4)) return -1;
    size_t n = (size_t)w * h;
    uint8_t *X = (uint8_t *)malloc(n), *Cx = NULL, *Dx = NULL;
    if (!X) return -1;
    for (size_t p = 0; p < n; ++p) X[p] = in[p] ? 1 : 0;
    if (C) {
        Cx = (uint8_t *)malloc(n);
        if (!Cx) { free(X); return -1; }
        for (size_t p = 0; p < n; ++p) Cx[p] = C[p] && X[p];
    }
    if (D) {
        Dx = (uint8_t *)malloc(n);
        if (!Dx) { free(X); free(Cx); return -1; }
        for (size_t p = 0; p < n; ++p) Dx[p] = D[p] && !X[p];
    }
    int rc = 0;
    for (int r = 1; r <= rmax && rc == 0; ++r) {
        rc = hasf_oracle_hc(X, Cx, w, h, r, conn, st);
        if (rc == 0) rc = hasf_oracle_hf(X, Dx, w, h, r, conn, st);
    }
    if (rc == 0) memcpy(out, X, n);
    free(X);
    free(Cx);
    free(Dx);
    return rc;
}

/* HASF run to stability: the order of the filter is not given; steps
 * r = 1, 2, ... (each HC_r^C then HF_r^D, as in hasf_oracle_hasf) are applied
 * until one leaves the image unchanged, at most rcap steps.  This is the
 * reading taken of the unbounded radius ("r = infinity") of Table 1.
 * out receives the image after the last step applied.  Returns the radius of
 * the step that changed nothing (the image is a fixed point of that step),
 * 0 if step rcap still changed the image, or -1 on bad arguments. */
int hasf_oracle_hasf_stable(const uint8_t *in, const uint8_t *C, const uint8_t *D, int w,
                            int h, int rcap, int conn, uint8_t *out, hasf_oracle_stats *st)
{
    if (w < 1 || h < 1 || rcap < 1 || (conn != 8 && conn != 4)) return -1;
    size_t n = (size_t)w * h;
    uint8_t *X = (uint8_t *)malloc(n), *prev = (uint8_t *)malloc(n), *Cx = NULL, *Dx = NULL;
    if (!X || !prev) { free(X); free(prev); return -1; }
    for (size_t p = 0; p < n; ++p) X[p] = in[p] ? 1 : 0;
    if (C) {
        Cx = (uint8_t *)malloc(n);
        if (!Cx) { free(X); free(prev); return -1; }
        for (size_t p = 0; p < n; ++p) Cx[p] = C[p] && X[p];
    }
    if (D) {
        Dx = (uint8_t *)malloc(n);
        if (!Dx) { free(X); free(prev); free(Cx); return -1; }
        for (size_t p = 0; p < n; ++p) Dx[p] = D[p] && !X[p];
    }
    int result = 0;
    for (int r = 1; r <= rcap; ++r) {
        memcpy(prev, X, n);
        if (hasf_oracle_hc(X, Cx, w, h, r, conn, st) != 0 ||
            hasf_oracle_hf(X, Dx, w, h, r, conn, st) != 0) {
            result = -1;
            break;
        }
        if (memcmp(prev, X, n) == 0) {
            result = r;
            break;
        }
    }
    if (result >= 0) memcpy(out, X, n);
    free(X);
    free(prev);
    free(Cx);
    free(Dx);
    return result;
}

/* Size of the statistics record, so that callers can check their layout. */
int hasf_oracle_stats_size(void) { return (int)sizeof(hasf_oracle_stats); }
