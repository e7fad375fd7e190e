/*
 * Multi-core CPU baseline of the uniform-grid build: the oracle's loops run
 * under OpenMP on every host core.  TEST AND BENCHMARK INFRASTRUCTURE ONLY,
 * like the oracle it is built with: bench.py times it as a CPU reference
 * point and the tests check it against the oracle.  It is not part of the
 * product path and shares no code with the CUDA library.
 *
 * The steps are the oracle's own (or_bounds, or_plan, or_cell_boxes compute
 * the boxes, the grid metadata and the cell counts V); the placement is the
 * counting placement of or_grid_counting split by z-slabs of cells (cell ids
 * are z-major, so a slab is a contiguous id range that one thread owns):
 *   1. each slab counts its cells' pairs, visiting the objects whose box
 *      meets the slab (objects in ascending order, no atomics);
 *   2. an exclusive scan over all cells -> G (two-pass, per-thread blocks);
 *   3. each slab places its pairs the same way, in ascending object order,
 *      which is the stable order of Algorithm 1's radix sort.
 * The result equals the oracle's grid bit for bit.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>

int or_bounds(const float *verts, int64_t nverts, const int32_t *tris, int64_t n, float lo[3], float hi[3]);
int or_plan(const float lo[3], const float hi[3], int64_t n, float lambda, int32_t res[3], float scale[3],
            int64_t *ncells);
int or_cell_boxes(const float *verts, const int32_t *tris, int64_t n, const float lo[3], const float scale[3],
                  const int32_t res[3], int32_t *clo, int32_t *chi, int64_t *V);

#define CP_OK 0
#define CP_EINVAL (-1)
#define CP_ENOMEM (-2)
#define CP_EOVERFLOW (-3)

/* Sets and returns the number of threads OpenMP uses (nthreads <= 0: every
 * host core). */
int cp_threads(int nthreads)
{
    omp_set_num_threads(nthreads > 0 ? nthreads : omp_get_num_procs());
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        t = omp_get_num_threads();
    }
    return t;
}

/* The whole build.  G must hold ncells + 1 entries and refs refs_cap; the
 * sizes come back in *ncells_out / *nrefs_out (OR_EOVERFLOW-style error if
 * refs_cap is too small: call with refs_cap = 0 to size, then again). */
int cp_build_grid(const float *verts, int64_t nverts, const int32_t *tris, int64_t n, float lambda,
                  int32_t *G, int64_t G_cap, int32_t *refs, int64_t refs_cap, int64_t *ncells_out,
                  int64_t *nrefs_out)
{
    float lo[3], hi[3], scale[3];
    int32_t res[3];
    int64_t ncells = 0;
    int rc = or_bounds(verts, nverts, tris, n, lo, hi);
    if (rc) return rc;
    rc = or_plan(lo, hi, n, lambda, res, scale, &ncells);
    if (rc) return rc;
    *ncells_out = ncells;
    int32_t *clo = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(n > 0 ? n : 1));
    int32_t *chi = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(n > 0 ? n : 1));
    int64_t *V = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cnt = NULL;
    if (!clo || !chi || !V) { rc = CP_ENOMEM; goto done; }
    /* boxes and V, objects in parallel chunks */
#pragma omp parallel
    {
        int nt = omp_get_num_threads(), t = omp_get_thread_num();
        int64_t i0 = n * t / nt, i1 = n * (t + 1) / nt;
        if (i1 > i0) or_cell_boxes(verts, tris + 3 * i0, i1 - i0, lo, scale, res, clo + 3 * i0, chi + 3 * i0, V + i0);
    }
    int64_t NO = 0;
#pragma omp parallel for reduction(+ : NO)
    for (int64_t i = 0; i < n; ++i) NO += V[i];
    *nrefs_out = NO;
    if (NO > INT32_MAX) { rc = CP_EOVERFLOW; goto done; }
    if (G_cap < ncells + 1 || refs_cap < NO) { rc = CP_EOVERFLOW; goto done; }
    cnt = (int64_t *)calloc((size_t)ncells + 1, sizeof(int64_t));
    if (!cnt) { rc = CP_ENOMEM; goto done; }
    {
        const int nt = omp_get_max_threads();
        const int64_t rz = res[2], rxy = (int64_t)res[0] * res[1];
        const int64_t nslabs = rz < 8 * (int64_t)nt ? rz : 8 * (int64_t)nt;
        /* 1. per-cell counts, slab by slab */
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t sl = 0; sl < nslabs; ++sl) {
            const int32_t z0 = (int32_t)(rz * sl / nslabs), z1 = (int32_t)(rz * (sl + 1) / nslabs);
            for (int64_t i = 0; i < n; ++i) {
                const int32_t *l = &clo[3 * i], *h = &chi[3 * i];
                const int32_t za = l[2] > z0 ? l[2] : z0, zb = h[2] < z1 - 1 ? h[2] : z1 - 1;
                for (int32_t z = za; z <= zb; ++z)
                    for (int32_t y = l[1]; y <= h[1]; ++y)
                        for (int32_t x = l[0]; x <= h[0]; ++x) cnt[x + res[0] * (int64_t)y + rxy * z] += 1;
            }
        }
        /* 2. exclusive scan -> G, then cnt becomes each cell's cursor */
        int64_t *part = (int64_t *)calloc((size_t)nt + 1, sizeof(int64_t));
        if (!part) { rc = CP_ENOMEM; goto done; }
#pragma omp parallel num_threads(nt)
        {
            const int t = omp_get_thread_num(), nth = omp_get_num_threads();
            const int64_t c0 = (ncells + 1) * t / nth, c1 = (ncells + 1) * (t + 1) / nth;
            int64_t s = 0;
            for (int64_t c = c0; c < c1; ++c) s += cnt[c];
            part[t + 1] = s;
#pragma omp barrier
#pragma omp single
            for (int k = 1; k <= nth; ++k) part[k] += part[k - 1];
            s = part[t];
            for (int64_t c = c0; c < c1; ++c) {
                const int64_t v = cnt[c];
                cnt[c] = s;
                G[c] = (int32_t)s;
                s += v;
            }
        }
        free(part);
        /* 3. placement, slab by slab, objects ascending */
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t sl = 0; sl < nslabs; ++sl) {
            const int32_t z0 = (int32_t)(rz * sl / nslabs), z1 = (int32_t)(rz * (sl + 1) / nslabs);
            for (int64_t i = 0; i < n; ++i) {
                const int32_t *l = &clo[3 * i], *h = &chi[3 * i];
                const int32_t za = l[2] > z0 ? l[2] : z0, zb = h[2] < z1 - 1 ? h[2] : z1 - 1;
                for (int32_t z = za; z <= zb; ++z)
                    for (int32_t y = l[1]; y <= h[1]; ++y)
                        for (int32_t x = l[0]; x <= h[0]; ++x) refs[cnt[x + res[0] * (int64_t)y + rxy * z]++] = (int32_t)i;
            }
        }
    }
done:
    free(clo);
    free(chi);
    free(V);
    free(cnt);
    return rc;
}
