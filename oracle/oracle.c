/*
 * CPU oracle for parallel uniform-grid construction ("BuildParallelGrid",
 * Algorithm 1 of Costa, Pereira, Jorge: "Building An Efficient Grid On GPU").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its Python binding) never calls into it, and the two
 * share no code: this file is plain sequential C, compiled with
 * -O2 -ffp-contract=off (no FMA contraction, no fast-math, no FTZ).
 *
 * What it computes (Sec. 3):
 *   boxes   per-triangle world AABB (min/max of its 3 vertices) and the scene
 *           bounds, their union;
 *   M       grid metadata: a resolution per axis from the density rule
 *           res_a = ceil(e_a * cbrt(lambda * N / volume)) (the paper leaves
 *           the cell-size heuristic open, Sec. 6), and scale_a = res_a / e_a;
 *   V       CountCells: cells covered by each object's box, in grid
 *           coordinates with inclusive hi (GlobalCoords, Sec. 3);
 *   NO, V   ExclusiveSum of V;
 *   O       MakeObjectIds (boundary markers) then InclusiveSum;
 *   C       SegmentedExclusiveSum of ones, then MakeCellIds via GlobalCoords;
 *   C, O    RadixSort of the (cell, object) pairs by cell (stable);
 *   G       RunLengthEncode(C), NonEmptyCells, ExclusiveSum -> compact grid.
 *
 * Readings where the paper is silent (each is also listed in the design
 * notes): the cell of a coordinate p on axis a is floor((p - lo_a) * scale_a)
 * with both operations rounded separately in FP32, clamped to [0, res_a - 1]
 * (NaN -> 0); cell ids are linearised x fastest: x + res_x * (y + res_y * z);
 * an axis of zero extent gets res 1 and scale 0 and the density root is taken
 * over the remaining axes; G has ncells + 1 entries with G[ncells] = NO.
 *
 * Besides the literal Algorithm 1 chain, the file holds two independent
 * restatements of the same grid used to pin it: a brute-force per-cell test
 * of every object box (tiny scenes) and a counting placement that visits each
 * object's box cells in ascending object order (any size).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_EOVERFLOW (-3)

#define OR_RES_MAX 65535

/* ---- boxes: per-triangle AABB and scene bounds (Sec. 3, "boxes") --------- */

/* Validates every vertex index and coordinate the triangles reference and
 * returns the union of the triangle boxes.  n == 0 gives lo = hi = 0.
 * A bound equal to zero is reported as +0.0 whichever sign of zero the
 * vertices carry (the paper does not distinguish them; -0.0 + 0.0 is +0.0
 * in round-to-nearest, every other value is unchanged).  The grid does not
 * depend on the sign: cell coordinates of +-0 offsets are 0 either way. */
int or_bounds(const float *verts, int64_t nverts, const int32_t *tris, int64_t n,
              float lo[3], float hi[3])
{
    if (n < 0 || nverts < 0) return OR_EINVAL;
    for (int a = 0; a < 3; ++a) { lo[a] = 0.0f; hi[a] = 0.0f; }
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) {
            int32_t vi = tris[3 * i + k];
            if (vi < 0 || (int64_t)vi >= nverts) return OR_EINVAL;
            for (int a = 0; a < 3; ++a) {
                float p = verts[3 * (int64_t)vi + a];
                if (!isfinite(p)) return OR_EINVAL;
                if (i == 0 && k == 0) { lo[a] = p; hi[a] = p; }
                if (p < lo[a]) lo[a] = p;
                if (p > hi[a]) hi[a] = p;
            }
        }
    }
    for (int a = 0; a < 3; ++a) {
        lo[a] = lo[a] + 0.0f;
        hi[a] = hi[a] + 0.0f;
    }
    return OR_OK;
}

/* ---- M: grid resolution and world-to-cell scale -------------------------- */

int or_plan(const float lo[3], const float hi[3], int64_t n, float lambda,
            int32_t res[3], float scale[3], int64_t *ncells)
{
    if (n < 0 || !isfinite(lambda) || !(lambda > 0.0f)) return OR_EINVAL;
    float e[3];
    int d = 0;
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) {
        e[a] = hi[a] - lo[a];
        res[a] = 1;
        scale[a] = 0.0f;
        if (n > 0 && e[a] > 0.0f) { ++d; vol = vol * (double)e[a]; }
    }
    if (d > 0) {
        double q = ((double)lambda * (double)n) / vol;
        double k = (d == 3) ? cbrt(q) : (d == 2) ? sqrt(q) : q;
        for (int a = 0; a < 3; ++a) {
            if (!(e[a] > 0.0f)) continue;
            double r = ceil((double)e[a] * k);
            if (!(r >= 1.0)) r = 1.0;
            if (r > (double)OR_RES_MAX) r = (double)OR_RES_MAX;
            res[a] = (int32_t)r;
            scale[a] = (float)res[a] / e[a];
        }
    }
    int64_t nc = (int64_t)res[0] * (int64_t)res[1] * (int64_t)res[2];
    *ncells = nc;
    if (nc > INT32_MAX) return OR_EOVERFLOW;
    return OR_OK;
}

/* ---- CountCells (Algorithm 1) -------------------------------------------- */

/* Grid coordinate of world value p on one axis. */
static int32_t or_cell_coord(float p, float lo, float scale, int32_t res)
{
    float t = p - lo;          /* rounded to FP32 */
    float u = t * scale;       /* rounded to FP32, separately */
    if (isnan(u)) return 0;
    float f = floorf(u);
    if (f < 0.0f) return 0;
    if (f > (float)(res - 1)) return res - 1;
    return (int32_t)f;
}

/* Per object: its box in grid coordinates (clo, chi inclusive, [n][3]) and
 * V = m_x * m_y * m_z with m = chi - clo + 1.  Inputs must have passed
 * or_bounds. */
int or_cell_boxes(const float *verts, const int32_t *tris, int64_t n,
                  const float lo[3], const float scale[3], const int32_t res[3],
                  int32_t *clo, int32_t *chi, int64_t *V)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t cnt = 1;
        for (int a = 0; a < 3; ++a) {
            float bl = 0.0f, bh = 0.0f;
            for (int k = 0; k < 3; ++k) {
                float p = verts[3 * (int64_t)tris[3 * i + k] + a];
                if (k == 0 || p < bl) bl = p;
                if (k == 0 || p > bh) bh = p;
            }
            int32_t cl = or_cell_coord(bl, lo[a], scale[a], res[a]);
            int32_t ch = or_cell_coord(bh, lo[a], scale[a], res[a]);
            clo[3 * i + a] = cl;
            chi[3 * i + a] = ch;
            cnt *= (int64_t)(ch - cl + 1);
        }
        V[i] = cnt;
    }
    return OR_OK;
}

/* ---- ExclusiveSum (Algorithm 1) ------------------------------------------ */

int or_exclusive_sum(const int64_t *V, int64_t n, int64_t *offsets, int64_t *total)
{
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i) {
        offsets[i] = s;
        s += V[i];
        if (s > INT32_MAX) { *total = s; return OR_EOVERFLOW; }
    }
    *total = s;
    return OR_OK;
}

/* ---- MakeObjectIds, InclusiveSum, SegmentedExclusiveSum, MakeCellIds ----- */

/* GlobalCoords (Sec. 3): relative cell offset rid inside a box whose extent
 * is m -> global grid coordinates (x fastest, then y, then z). */
static void or_global_coords(const int32_t lo[3], const int32_t hi[3], int64_t rid,
                             int32_t out[3])
{
    int64_t mx = (int64_t)hi[0] - lo[0] + 1;
    int64_t my = (int64_t)hi[1] - lo[1] + 1;
    int64_t z = rid / (mx * my);
    int64_t y = (rid - z * mx * my) / mx;
    int64_t x = rid - mx * (y + my * z);
    out[0] = lo[0] + (int32_t)x;
    out[1] = lo[1] + (int32_t)y;
    out[2] = lo[2] + (int32_t)z;
}

static int32_t or_linear_cell(const int32_t g[3], const int32_t res[3])
{
    return (int32_t)((int64_t)g[0] + (int64_t)res[0] * ((int64_t)g[1] + (int64_t)res[1] * (int64_t)g[2]));
}

/* The object-order pair lists of Fig. 4a/4b, built with the literal steps of
 * Algorithm 1: O <- 0; O[V[i]] <- 1 for i in ]0, nobjs[ (V holding the
 * exclusive offsets); O <- InclusiveSum(O); C <- 1;
 * C <- SegmentedExclusiveSum(C) with boundaries where O[j] != O[j-1];
 * C <- GlobalCoords(box[O[j]], C[j]) linearised. */
int or_object_order_pairs(const int32_t *clo, const int32_t *chi, const int64_t *offsets,
                          int64_t n, int64_t NO, const int32_t res[3],
                          int32_t *C, int32_t *O)
{
    if (NO == 0) return OR_OK;
    /* MakeObjectIds */
    for (int64_t j = 0; j < NO; ++j) O[j] = 0;
    for (int64_t i = 1; i < n; ++i) O[offsets[i]] = 1;
    /* InclusiveSum(O) */
    for (int64_t j = 1; j < NO; ++j) O[j] = O[j] + O[j - 1];
    /* C <- 1; SegmentedExclusiveSum(C) */
    for (int64_t j = 0; j < NO; ++j) C[j] = 1;
    int32_t run = 0;
    for (int64_t j = 0; j < NO; ++j) {
        int32_t one = C[j];
        if (j == 0 || O[j] != O[j - 1]) run = 0;
        C[j] = run;
        run += one;
    }
    /* MakeCellIds */
    for (int64_t j = 0; j < NO; ++j) {
        int32_t g[3];
        int64_t o = O[j];
        or_global_coords(&clo[3 * o], &chi[3 * o], C[j], g);
        C[j] = or_linear_cell(g, res);
    }
    return OR_OK;
}

/* ---- RadixSort(C, O): a stable sort by cell id ---------------------------- */

typedef struct { int32_t c, o; int64_t j; } or_pair;

static int or_pair_cmp(const void *pa, const void *pb)
{
    const or_pair *a = (const or_pair *)pa, *b = (const or_pair *)pb;
    if (a->c != b->c) return a->c < b->c ? -1 : 1;
    return a->j < b->j ? -1 : (a->j > b->j ? 1 : 0); /* original position: stable */
}

int or_sort_pairs(int32_t *C, int32_t *O, int64_t NO)
{
    if (NO == 0) return OR_OK;
    or_pair *p = (or_pair *)malloc((size_t)NO * sizeof(or_pair));
    if (!p) return OR_ENOMEM;
    for (int64_t j = 0; j < NO; ++j) { p[j].c = C[j]; p[j].o = O[j]; p[j].j = j; }
    qsort(p, (size_t)NO, sizeof(or_pair), or_pair_cmp);
    for (int64_t j = 0; j < NO; ++j) { C[j] = p[j].c; O[j] = p[j].o; }
    free(p);
    return OR_OK;
}

/* ---- RunLengthEncode, NonEmptyCells, ExclusiveSum -> G ------------------- */

/* G has ncells + 1 entries; G[c] is where cell c's object ids start in the
 * sorted O and G[ncells] = NO closes the last cell. */
int or_ranges(const int32_t *Csorted, int64_t NO, int64_t ncells, int32_t *G)
{
    /* RunLengthEncode(C): unique cells and their run lengths */
    int32_t *uniq = (int32_t *)malloc((size_t)(NO > 0 ? NO : 1) * sizeof(int32_t));
    int64_t *counts = (int64_t *)malloc((size_t)(NO > 0 ? NO : 1) * sizeof(int64_t));
    if (!uniq || !counts) { free(uniq); free(counts); return OR_ENOMEM; }
    int64_t nonEmpty = 0;
    for (int64_t j = 0; j < NO; ++j) {
        if (j == 0 || Csorted[j] != Csorted[j - 1]) {
            uniq[nonEmpty] = Csorted[j];
            counts[nonEmpty] = 0;
            ++nonEmpty;
        }
        counts[nonEmpty - 1] += 1;
    }
    /* G <- 0; NonEmptyCells */
    int64_t *g = (int64_t *)calloc((size_t)ncells + 1, sizeof(int64_t));
    if (!g) { free(uniq); free(counts); return OR_ENOMEM; }
    for (int64_t r = 0; r < nonEmpty; ++r) {
        if (uniq[r] < 0 || uniq[r] >= ncells) { free(uniq); free(counts); free(g); return OR_EINVAL; }
        g[uniq[r]] = counts[r];
    }
    /* ExclusiveSum(G) over ncells + 1 entries */
    int64_t s = 0;
    for (int64_t c = 0; c <= ncells; ++c) {
        int64_t v = g[c];
        G[c] = (int32_t)s;
        s += v;
    }
    free(uniq); free(counts); free(g);
    return OR_OK;
}

/* ---- independent restatements used to pin the chain above ---------------- */

/* Counting placement: G[c] = number of (object, cell) incidences with cell
 * < c, and each cell's list is filled by visiting objects in ascending id and
 * each object's box cells.  refs must hold NO entries. */
int or_grid_counting(const int32_t *clo, const int32_t *chi, int64_t n, const int32_t res[3],
                     int64_t ncells, int32_t *G, int32_t *refs)
{
    int64_t *cnt = (int64_t *)calloc((size_t)ncells + 1, sizeof(int64_t));
    if (!cnt) return OR_ENOMEM;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t *l = &clo[3 * i], *h = &chi[3 * i];
        for (int32_t z = l[2]; z <= h[2]; ++z)
            for (int32_t y = l[1]; y <= h[1]; ++y)
                for (int32_t x = l[0]; x <= h[0]; ++x) {
                    int32_t g3[3] = {x, y, z};
                    cnt[or_linear_cell(g3, res)] += 1;
                }
    }
    int64_t s = 0;
    for (int64_t c = 0; c <= ncells; ++c) {
        int64_t v = cnt[c];
        cnt[c] = s;
        G[c] = (int32_t)s;
        s += v;
    }
    for (int64_t i = 0; i < n; ++i) {
        const int32_t *l = &clo[3 * i], *h = &chi[3 * i];
        for (int32_t z = l[2]; z <= h[2]; ++z)
            for (int32_t y = l[1]; y <= h[1]; ++y)
                for (int32_t x = l[0]; x <= h[0]; ++x) {
                    int32_t g3[3] = {x, y, z};
                    int32_t c = or_linear_cell(g3, res);
                    refs[cnt[c]++] = (int32_t)i;
                }
    }
    free(cnt);
    return OR_OK;
}

/* Brute force over every (cell, object): an object is listed in cell
 * (x, y, z) iff clo <= (x, y, z) <= chi on all three axes.  O(ncells * n):
 * tiny scenes only.  refs must hold refs_cap entries; returns OR_EOVERFLOW if
 * the grid has more. */
int or_grid_bruteforce(const int32_t *clo, const int32_t *chi, int64_t n, const int32_t res[3],
                       int32_t *G, int32_t *refs, int64_t refs_cap, int64_t *nrefs)
{
    int64_t k = 0;
    int64_t c = 0;
    for (int32_t z = 0; z < res[2]; ++z)
        for (int32_t y = 0; y < res[1]; ++y)
            for (int32_t x = 0; x < res[0]; ++x, ++c) {
                G[c] = (int32_t)k;
                for (int64_t i = 0; i < n; ++i) {
                    const int32_t *l = &clo[3 * i], *h = &chi[3 * i];
                    if (l[0] <= x && x <= h[0] && l[1] <= y && y <= h[1] && l[2] <= z && z <= h[2]) {
                        if (k >= refs_cap) return OR_EOVERFLOW;
                        refs[k++] = (int32_t)i;
                    }
                }
            }
    G[c] = (int32_t)k;
    *nrefs = k;
    return OR_OK;
}

/* ---- False-intersection culling (Sec. 6, future work) ----------------------
 *
 * The box placement above lists an object in every cell of its bounding box,
 * so a long diagonal triangle lands in many cells it does not touch.  The
 * paper names a triangle/cell overlap test ahead of the sort as future work.
 * This is that test, with one fixed reading:
 *
 *   grid-space vertex  q_k = min((v_k - lo) * scale, res) per axis: the two
 *                      FP32 operations of the cell mapping, so floor(q) is
 *                      the vertex's cell, and the clamp to the grid's far
 *                      face that the mapping applies to cells (scale =
 *                      res / e rounded to FP32 can put the far face's vertex
 *                      up to res 2^-23 beyond res, outside the last cell);
 *   cell (x, y, z)     the closed unit cube centred at c = (x, y, z) + 1/2;
 *   local vertex       w_k = q_k - c;
 *   edges              e_0 = q_1 - q_0, e_1 = q_2 - q_1, e_2 = q_0 - q_2;
 *   axes               the normal n = e_0 x e_1 and, for each edge e and unit
 *                      axis, unit x e: (0, -e_z, e_y), (e_z, 0, -e_x) and
 *                      (-e_y, e_x, 0) (separating-axis theorem for a
 *                      triangle against a box);
 *   projection         p_k = (a_x w_kx + a_y w_ky) + a_z w_kz;
 *   box radius         S = (|a_x| + |a_y|) + |a_z|, r = S / 2;
 *   slack              t = W 2^-16 + 2^-10 with W = max_{k,a} |w_ka|, and
 *                      R = r + S t;
 *   separated          min_k p_k > R or max_k p_k < -R.
 *
 * A pair is dropped iff one of the ten axes separates.  Every product, sum and
 * difference is a single FP32 operation in the order written (no fused
 * multiply-add), so the decision is exact and machine-independent.  The
 * rounding error of p_k is a few units of 2^-24 S W, far below the slack
 * S t, so a triangle that touches the closed cell is never dropped, while a
 * cell that an axis separates by more than about t cell widths always is.
 * The three face normals are not tested: each cell of the object's cell box
 * already meets the triangle's extent along x, y and z.
 *
 * Both triangle and cell are the grid-space ones; the world-space triangle
 * differs from the grid-space one by the rounding of the cell mapping only. */

#define OR_SLACK_REL 0x1p-16f
#define OR_SLACK_ABS 0x1p-10f

/* 1 if the triangle with grid-space vertices q (q[3k + a]) is separated from
 * cell (x, y, z), else 0. */
int or_tri_cell_separated(const float *q, int32_t x, int32_t y, int32_t z)
{
    const float c[3] = {(float)x + 0.5f, (float)y + 0.5f, (float)z + 0.5f};
    float w[3][3];
    float W = 0.0f;
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a) {
            w[k][a] = q[3 * k + a] - c[a];
            W = fmaxf(W, fabsf(w[k][a]));
        }
    const float t = W * OR_SLACK_REL + OR_SLACK_ABS;
    float e[3][3];
    for (int a = 0; a < 3; ++a) {
        e[0][a] = q[3 + a] - q[a];
        e[1][a] = q[6 + a] - q[3 + a];
        e[2][a] = q[a] - q[6 + a];
    }
    float ax[10][3];
    ax[0][0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
    ax[0][1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
    ax[0][2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
    for (int j = 0; j < 3; ++j) {
        ax[1 + j][0] = 0.0f;
        ax[1 + j][1] = -e[j][2];
        ax[1 + j][2] = e[j][1];
        ax[4 + j][0] = e[j][2];
        ax[4 + j][1] = 0.0f;
        ax[4 + j][2] = -e[j][0];
        ax[7 + j][0] = -e[j][1];
        ax[7 + j][1] = e[j][0];
        ax[7 + j][2] = 0.0f;
    }
    for (int s = 0; s < 10; ++s) {
        const float *a = ax[s];
        float pmin = 0.0f, pmax = 0.0f;
        for (int k = 0; k < 3; ++k) {
            float p = a[0] * w[k][0] + a[1] * w[k][1];
            p = p + a[2] * w[k][2];
            if (k == 0 || p < pmin) pmin = p;
            if (k == 0 || p > pmax) pmax = p;
        }
        const float S = (fabsf(a[0]) + fabsf(a[1])) + fabsf(a[2]);
        const float R = 0.5f * S + S * t;
        if (pmin > R || pmax < -R) return 1;
    }
    return 0;
}

/* The object-order pair lists of the box placement with the separated pairs
 * removed: objects ascending, each object's box cells in GlobalCoords order
 * (x fastest), a cell kept iff or_tri_cell_separated says 0.  kept[i] gets
 * object i's kept count.  C, O hold cap entries; *NOk gets the number kept
 * (OR_EOVERFLOW if it would pass cap or INT32_MAX).  Inputs must have passed
 * or_bounds, and clo / chi come from or_cell_boxes on the same plan. */
int or_cull_pairs(const float *verts, const int32_t *tris, int64_t n, const float lo[3],
                  const float scale[3], const int32_t res[3], const int32_t *clo, const int32_t *chi,
                  int64_t cap, int32_t *C, int32_t *O, int64_t *kept, int64_t *NOk)
{
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        float q[9];
        for (int v = 0; v < 3; ++v)
            for (int a = 0; a < 3; ++a) {
                float t = verts[3 * (int64_t)tris[3 * i + v] + a] - lo[a];
                float u = t * scale[a];
                q[3 * v + a] = u > (float)res[a] ? (float)res[a] : u;
            }
        const int32_t *l = &clo[3 * i], *h = &chi[3 * i];
        int64_t ki = 0;
        for (int32_t z = l[2]; z <= h[2]; ++z)
            for (int32_t y = l[1]; y <= h[1]; ++y)
                for (int32_t x = l[0]; x <= h[0]; ++x) {
                    if (or_tri_cell_separated(q, x, y, z)) continue;
                    if (k >= cap || k >= INT32_MAX) { *NOk = k; return OR_EOVERFLOW; }
                    int32_t g3[3] = {x, y, z};
                    C[k] = or_linear_cell(g3, res);
                    O[k] = (int32_t)i;
                    ++k;
                    ++ki;
                }
        kept[i] = ki;
    }
    *NOk = k;
    return OR_OK;
}

/* Stable counting placement of object-order pairs: G[c] = number of pairs
 * with cell < c (G[ncells] = NO), refs = the objects in cell order, ties in
 * input order.  A second, independent route to RadixSort + the range steps
 * for pairs given as lists. */
int or_place_stable(const int32_t *C, const int32_t *O, int64_t NO, int64_t ncells, int32_t *G,
                    int32_t *refs)
{
    int64_t *cnt = (int64_t *)calloc((size_t)ncells + 1, sizeof(int64_t));
    if (!cnt) return OR_ENOMEM;
    for (int64_t j = 0; j < NO; ++j) {
        if (C[j] < 0 || (int64_t)C[j] >= ncells) { free(cnt); return OR_EINVAL; }
        cnt[C[j]] += 1;
    }
    int64_t s = 0;
    for (int64_t c = 0; c <= ncells; ++c) {
        int64_t v = cnt[c];
        cnt[c] = s;
        G[c] = (int32_t)s;
        s += v;
    }
    for (int64_t j = 0; j < NO; ++j) refs[cnt[C[j]]++] = O[j];
    free(cnt);
    return OR_OK;
}
