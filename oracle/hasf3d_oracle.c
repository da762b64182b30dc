/*
 * hasf3d_oracle.c -- CPU oracle for the three-dimensional HASF.
 *
 * TEST INFRASTRUCTURE ONLY, like hasf_oracle.c: loaded by the tests and the
 * CPU legs of the benchmark, never by the CUDA library, and sharing no code
 * with it.
 *
 * The paper states the method for 2D images and notes (Sec. 1) that it
 * applies to 3D images as well.  This file is that extension, written with
 * the same structure as the 2D oracle:
 *  - a volume is w x h x d bytes, x fastest: voxel (x, y, z) at
 *    [(z*h + y)*w + x]; non-zero = object; everything outside the box is
 *    background, fixed forever;
 *  - adjacency pair (26, 6): 26-connected object, 6-connected background;
 *  - a voxel x is simple (the 3D counterpart of T = 1 and Tbar = 1 of Sec. 2)
 *    when the object voxels of its 26-neighbourhood form exactly one
 *    26-connected component, and the background voxels of its
 *    18-neighbourhood that are 6-connected to one of x's six face neighbours
 *    form exactly one 6-connected component (the topological numbers of
 *    Bertrand and Malandain);
 *  - distances are squared Euclidean, clamped at r^2 + 1 (every candidate of
 *    every operator of HC_r / HF_r has priority <= r^2, the argument of the
 *    2D oracle carries over unchanged);
 *  - H / *H: levels (distinct candidate priorities) ascending; at each level
 *    rounds until a round changes nothing; a round visits the eight
 *    subfields (x mod 2, y mod 2, z mod 2) in the order s = 0..7 with
 *    (x, y, z) parities (s & 1, (s >> 1) & 1, s >> 2), each in raster order
 *    (z, then y, then x).  Two voxels of one subfield differ by an even amount
 *    in every coordinate, so they are never 26-adjacent and the order inside a
 *    subfield does not matter;
 *  - HC_r^C, HF_r^D and HASF as eqs. (i), (ii) of Sec. 2 with B_r the ball
 *    |v|^2 <= r^2.
 *
 * Parity status: the simple-voxel test is pinned by component labelling, the
 * distance map by brute force, the operators by invariants, a solid box and
 * a hand-worked thinning, and the composition of the filter (radii
 * ascending, cutting before filling) by the alternating sequential filter by
 * ball unions, which it equals on topologically trivial boxes with slabs and
 * notches.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Cube positions: offset (dx, dy, dz) is position (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1). */
static void offs_of(int i, int *dx, int *dy, int *dz)
{
    *dx = i % 3 - 1;
    *dy = (i / 3) % 3 - 1;
    *dz = i / 9 - 1;
}

static int iabs(int v) { return v < 0 ? -v : v; }

/* Number of connected components of the positions in `members` (a bit set
 * over the 27 cube positions) under 26-adjacency (adj26 = 1) or 6-adjacency,
 * counting only the components that contain a position of `touch` (all
 * components if touch has every bit set).  Plain breadth-first search. */
static int count_components(uint32_t members, int adj26, uint32_t touch)
{
    uint32_t seen = 0;
    int count = 0;
    for (int s = 0; s < 27; ++s) {
        if (!((members >> s) & 1u) || ((seen >> s) & 1u)) continue;
        int queue[27], head = 0, tail = 0, touches = 0;
        queue[tail++] = s;
        seen |= 1u << s;
        while (head < tail) {
            int a = queue[head++];
            if ((touch >> a) & 1u) touches = 1;
            int ax, ay, az;
            offs_of(a, &ax, &ay, &az);
            for (int b = 0; b < 27; ++b) {
                if (!((members >> b) & 1u) || ((seen >> b) & 1u)) continue;
                int bx, by, bz;
                offs_of(b, &bx, &by, &bz);
                int ddx = iabs(ax - bx), ddy = iabs(ay - by), ddz = iabs(az - bz);
                int adjacent = adj26 ? (ddx <= 1 && ddy <= 1 && ddz <= 1)
                                     : (ddx + ddy + ddz == 1);
                if (!adjacent) continue;
                seen |= 1u << b;
                queue[tail++] = b;
            }
        }
        count += touches;
    }
    return count;
}

/* Simplicity of the centre voxel given its 3 x 3 x 3 neighbourhood `code`
 * (bit (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1) = object; the centre bit is
 * ignored). */
int hasf3d_oracle_simple(uint32_t code)
{
    uint32_t n26 = 0, n18 = 0, n6 = 0;
    for (int i = 0; i < 27; ++i) {
        int dx, dy, dz;
        offs_of(i, &dx, &dy, &dz);
        int l1 = iabs(dx) + iabs(dy) + iabs(dz);
        if (l1 == 0) continue;
        n26 |= 1u << i;
        if (l1 <= 2) n18 |= 1u << i;
        if (l1 == 1) n6 |= 1u << i;
    }
    uint32_t obj = code & n26;
    uint32_t bg18 = ~code & n18;
    int t26 = count_components(obj, 1, 0x7FFFFFFu);
    int t6 = count_components(bg18, 0, n6);
    return t26 == 1 && t6 == 1;
}

static uint32_t neighbour_code(const uint8_t *S, int w, int h, int d, int x, int y, int z)
{
    uint32_t code = 0;
    for (int i = 0; i < 27; ++i) {
        int dx, dy, dz;
        offs_of(i, &dx, &dy, &dz);
        int xx = x + dx, yy = y + dy, zz = z + dz;
        if (xx < 0 || yy < 0 || zz < 0 || xx >= w || yy >= h || zz >= d) continue;
        if (S[((size_t)zz * h + yy) * w + xx]) code |= 1u << i;
    }
    return code;
}

/* Squared distance from every voxel of the box to the nearest feature voxel,
 * clamped at r^2 + 1: the smallest |v|^2 <= r^2 such that p + v is a feature,
 * else r^2 + 1.  feat: non-zero = feature inside the box; outside the box
 * every point is a feature when outside_is_feature is set, none otherwise.
 * Plain search over the ball of radius r. */
int hasf3d_oracle_edt(const uint8_t *feat, int w, int h, int d, int outside_is_feature, int r,
                      int64_t *out)
{
    if (w < 1 || h < 1 || d < 1 || r < 0) return -1;
    int64_t cap = (int64_t)r * r + 1;
    for (int z = 0; z < d; ++z)
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                int64_t best = cap;
                for (int dz = -r; dz <= r; ++dz)
                    for (int dy = -r; dy <= r; ++dy)
                        for (int dx = -r; dx <= r; ++dx) {
                            int64_t n2 = (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz;
                            if (n2 >= best) continue;
                            int xx = x + dx, yy = y + dy, zz = z + dz;
                            int f;
                            if (xx < 0 || yy < 0 || zz < 0 || xx >= w || yy >= h || zz >= d)
                                f = outside_is_feature;
                            else
                                f = feat[((size_t)zz * h + yy) * w + xx] != 0;
                            if (f) best = n2;
                        }
                out[((size_t)z * h + y) * w + x] = best;
            }
    return 0;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* H (remove = 1) or *H (remove = 0) in 3D, in the order stated at the top.
 * K: points that must stay (thinning) or may be added (thickening). */
static int sweep3d(uint8_t *S, const uint8_t *K, const int64_t *prio, int w, int h, int d,
                   int remove)
{
    size_t n = (size_t)w * h * d;
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
        for (;;) {
            int changed = 0;
            for (int s = 0; s < 8; ++s) {
                int sx = s & 1, sy = (s >> 1) & 1, sz = s >> 2;
                for (int z = sz; z < d; z += 2)
                    for (int y = sy; y < h; y += 2)
                        for (int x = sx; x < w; x += 2) {
                            size_t p = ((size_t)z * h + y) * w + x;
                            int cand = remove ? (S[p] && !K[p]) : (!S[p] && K[p]);
                            if (!cand || prio[p] > level) continue;
                            if (hasf3d_oracle_simple(neighbour_code(S, w, h, d, x, y, z))) {
                                S[p] = (uint8_t)!remove;
                                changed = 1;
                            }
                        }
            }
            if (!changed) break;
        }
    }
    free(lv);
    return 0;
}

/* HC_r^C in 3D (eq. (i)): Y = H(X, eps_r(X) cup C), then *H(Y, delta_r(Y) cap X). */
static int hc3d(uint8_t *X, const uint8_t *C, int w, int h, int d, int r)
{
    size_t n = (size_t)w * h * d;
    int64_t *dist = (int64_t *)malloc(n * sizeof(int64_t));
    uint8_t *K = (uint8_t *)malloc(n), *bg = (uint8_t *)malloc(n);
    int rc = -1;
    if (!dist || !K || !bg) goto done;
    int64_t r2 = (int64_t)r * r;
    for (size_t p = 0; p < n; ++p) bg[p] = !X[p];
    if (hasf3d_oracle_edt(bg, w, h, d, 1, r, dist)) goto done;   /* to the complement of X */
    for (size_t p = 0; p < n; ++p) K[p] = (X[p] && dist[p] > r2) || (C && C[p]);
    if (sweep3d(X, K, dist, w, h, d, 1)) goto done;
    if (hasf3d_oracle_edt(X, w, h, d, 0, r, dist)) goto done;    /* to Y */
    /* V = delta_r(Y) cap X, X being the input kept in bg's complement */
    for (size_t p = 0; p < n; ++p) K[p] = dist[p] <= r2 && !bg[p];
    if (sweep3d(X, K, dist, w, h, d, 0)) goto done;
    rc = 0;
done:
    free(dist);
    free(K);
    free(bg);
    return rc;
}

/* HF_r^D in 3D (eq. (ii), W read as eps_r(Z) cup X): Z = *H(X, delta_r(X) minus D),
 * then H(Z, eps_r(Z) cup X). */
static int hf3d(uint8_t *X, const uint8_t *D, int w, int h, int d, int r)
{
    size_t n = (size_t)w * h * d;
    int64_t *dist = (int64_t *)malloc(n * sizeof(int64_t));
    uint8_t *K = (uint8_t *)malloc(n), *x0 = (uint8_t *)malloc(n), *bg = (uint8_t *)malloc(n);
    int rc = -1;
    if (!dist || !K || !x0 || !bg) goto done;
    int64_t r2 = (int64_t)r * r;
    memcpy(x0, X, n);
    if (hasf3d_oracle_edt(X, w, h, d, 0, r, dist)) goto done;    /* to X */
    for (size_t p = 0; p < n; ++p) K[p] = dist[p] <= r2 && !(D && D[p]);
    if (sweep3d(X, K, dist, w, h, d, 0)) goto done;
    for (size_t p = 0; p < n; ++p) bg[p] = !X[p];
    if (hasf3d_oracle_edt(bg, w, h, d, 1, r, dist)) goto done;   /* to the complement of Z */
    for (size_t p = 0; p < n; ++p) K[p] = (X[p] && dist[p] > r2) || x0[p];
    if (sweep3d(X, K, dist, w, h, d, 1)) goto done;
    rc = 0;
done:
    free(dist);
    free(K);
    free(x0);
    free(bg);
    return rc;
}

/* HASF_rmax^{C,D} of a volume: for r = 1..rmax, HC_r^C then HF_r^D.  C is
 * taken as C cap X and D as D minus X; either may be NULL.  out receives 0/1
 * bytes and may alias in.  Returns 0, or -1 on bad arguments. */
int hasf3d_oracle_hasf(const uint8_t *in, const uint8_t *C, const uint8_t *D, int w, int h,
                       int d, int rmax, uint8_t *out)
{
    if (w < 1 || h < 1 || d < 1 || rmax < 0) return -1;
    size_t n = (size_t)w * h * d;
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
        rc = hc3d(X, Cx, w, h, d, r);
        if (rc == 0) rc = hf3d(X, Dx, w, h, d, r);
    }
    if (rc == 0) memcpy(out, X, n);
    free(X);
    free(Cx);
    free(Dx);
    return rc;
}

/* The single operators, for the tests: H (thin = 1) or *H of S constrained by
 * K with the clamped priority of radius r (distance to the complement of S
 * for H, to S for *H). */
int hasf3d_oracle_operator(uint8_t *S, const uint8_t *K, int w, int h, int d, int r, int thin)
{
    size_t n = (size_t)w * h * d;
    int64_t *dist = (int64_t *)malloc(n * sizeof(int64_t));
    uint8_t *bg = (uint8_t *)malloc(n);
    int rc = -1;
    if (dist && bg) {
        for (size_t p = 0; p < n; ++p) bg[p] = !S[p];
        rc = thin ? hasf3d_oracle_edt(bg, w, h, d, 1, r, dist)
                  : hasf3d_oracle_edt(S, w, h, d, 0, r, dist);
        if (rc == 0) rc = sweep3d(S, K, dist, w, h, d, thin);
    }
    free(dist);
    free(bg);
    return rc;
}
