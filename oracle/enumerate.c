/*
 * FP64 CPU oracle: direct closed-triangle enumeration on the uv grid.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (Section 3.2 of arXiv:2506.10526):
 *   Eq. (iFT) / Eq. (iFT_I) define D and I as inverse Fourier transforms of
 *   W V and W N restricted to an annular ring.  Because the sum over image
 *   pixels of exp(-i (l1 + l2 + l3) . theta) vanishes unless the three grid
 *   points close, the numerator and denominator of the binned estimator
 *   Eq. (estimator_t) are (up to the same pixel-count factor) sums over all
 *   closed grid triangles U_g1 + U_g2 + U_g3 = 0 with U_gk in ring a_k, as the
 *   text after Eq. (estimator_t) states.  This file writes those sums out
 *   literally, in FP64, with no FFT:
 *
 *     num(i,j,l; nu1,nu2,nu3) = sum_{g1 in a_i, g2 in a_j, g3 = -g1-g2 in a_l}
 *                               X(g1,nu1) X(g2,nu2) X(g3,nu3),   X = W V
 *     den(i,j,l; nu1,nu2,nu3) = same sum of Y(g1,nu1) Y(g2,nu2) Y(g3,nu3),
 *                               Y = W N
 *     T(i,j,l)                = number of such ordered triangles
 *
 * Grid convention: arrays are centred, cell index c = (v + nt/2) * nt + (u + nt/2)
 * for integer u, v in [-nt/2, nt/2).  label[c] is the ring index of the cell or
 * -1 when the cell is not binned.  Complex data are split into re / im arrays.
 *
 * Per-channel data are laid out [nc][nt*nt] on input and transposed here to
 * [cell][nc] for locality.  OpenMP parallelises over ring triples, first
 * corners or sample points; per-thread accumulators are summed at the end.
 */
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n;
    int *u, *v, *cell;
} ring_cells;

static void free_rings(ring_cells *rc, int nb) {
    if (!rc) return;
    for (int m = 0; m < nb; ++m) {
        free(rc[m].u);
        free(rc[m].v);
        free(rc[m].cell);
    }
    free(rc);
}

/* Cell lists per ring, in increasing cell index. */
static ring_cells *build_rings(int nt, int nb, const int *label) {
    ring_cells *rc = (ring_cells *)calloc((size_t)nb, sizeof(ring_cells));
    if (!rc) return NULL;
    int ncell = nt * nt;
    for (int c = 0; c < ncell; ++c)
        if (label[c] >= 0 && label[c] < nb) rc[label[c]].n++;
    for (int m = 0; m < nb; ++m) {
        size_t n = (size_t)(rc[m].n > 0 ? rc[m].n : 1);
        rc[m].u = (int *)malloc(n * sizeof(int));
        rc[m].v = (int *)malloc(n * sizeof(int));
        rc[m].cell = (int *)malloc(n * sizeof(int));
        if (!rc[m].u || !rc[m].v || !rc[m].cell) {
            free_rings(rc, nb);
            return NULL;
        }
        rc[m].n = 0;
    }
    for (int c = 0; c < ncell; ++c) {
        int m = label[c];
        if (m < 0 || m >= nb) continue;
        int k = rc[m].n++;
        rc[m].u[k] = c % nt - nt / 2;
        rc[m].v[k] = c / nt - nt / 2;
        rc[m].cell[k] = c;
    }
    return rc;
}

/* Index of the cell at (u, v), or -1 when it lies outside the stored grid. */
static inline int cell_of(int nt, int u, int v) {
    int iu = u + nt / 2, iv = v + nt / 2;
    if (iu < 0 || iu >= nt || iv < 0 || iv >= nt) return -1;
    return iv * nt + iu;
}

/* [nc][ncell] -> [ncell][nc] */
static double *transpose_cc(const double *a, int nc, int ncell) {
    double *t = (double *)malloc((size_t)nc * (size_t)ncell * sizeof(double));
    if (!t) return NULL;
    for (int f = 0; f < nc; ++f)
        for (int c = 0; c < ncell; ++c) t[(size_t)c * nc + f] = a[(size_t)f * ncell + c];
    return t;
}

static int nthreads_or_default(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/*
 * Full channel cube for a list of ring triples.
 * xre, xim, y: [nc][nt*nt].  trip: [ntrip][3] = (i, j, l).
 * Outputs [ntrip][nc][nc][nc] (nu1 slowest, nu3 fastest) and tcount[ntrip].
 * Returns 0 on success, -1 on allocation failure.
 */
int orc_enumerate(int nt, int nc, int nb, const int *label, const double *xre,
                  const double *xim, const double *y, int ntrip, const int *trip,
                  double *num_re, double *num_im, double *den, long long *tcount,
                  int nthreads) {
    int ncell = nt * nt;
    ring_cells *rc = build_rings(nt, nb, label);
    double *tr = transpose_cc(xre, nc, ncell);
    double *ti = transpose_cc(xim, nc, ncell);
    double *ty = transpose_cc(y, nc, ncell);
    if (!rc || !tr || !ti || !ty) {
        free_rings(rc, nb);
        free(tr);
        free(ti);
        free(ty);
        return -1;
    }
    size_t cube = (size_t)nc * nc * nc;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads_or_default(nthreads))
    for (int t = 0; t < ntrip; ++t) {
        int ri = trip[3 * t], rj = trip[3 * t + 1], rl = trip[3 * t + 2];
        double *nr = num_re + (size_t)t * cube;
        double *ni = num_im + (size_t)t * cube;
        double *dn = den + (size_t)t * cube;
        memset(nr, 0, cube * sizeof(double));
        memset(ni, 0, cube * sizeof(double));
        memset(dn, 0, cube * sizeof(double));
        long long count = 0;
        if (ri < 0 || ri >= nb || rj < 0 || rj >= nb || rl < 0 || rl >= nb) {
            tcount[t] = 0;
            continue;
        }
        double *pr = (double *)malloc((size_t)nc * nc * sizeof(double));
        double *pi = (double *)malloc((size_t)nc * nc * sizeof(double));
        double *py = (double *)malloc((size_t)nc * nc * sizeof(double));
        if (!pr || !pi || !py) {
#pragma omp atomic write
            err = 1;
            free(pr);
            free(pi);
            free(py);
            continue;
        }
        const ring_cells *a = &rc[ri], *b = &rc[rj];
        for (int p = 0; p < a->n; ++p) {
            for (int q = 0; q < b->n; ++q) {
                int c3 = cell_of(nt, -a->u[p] - b->u[q], -a->v[p] - b->v[q]);
                if (c3 < 0 || label[c3] != rl) continue;
                ++count;
                const double *x1r = tr + (size_t)a->cell[p] * nc, *x1i = ti + (size_t)a->cell[p] * nc;
                const double *x2r = tr + (size_t)b->cell[q] * nc, *x2i = ti + (size_t)b->cell[q] * nc;
                const double *x3r = tr + (size_t)c3 * nc, *x3i = ti + (size_t)c3 * nc;
                const double *y1 = ty + (size_t)a->cell[p] * nc, *y2 = ty + (size_t)b->cell[q] * nc;
                const double *y3 = ty + (size_t)c3 * nc;
                /* pair products of the first two corners */
                for (int n1 = 0; n1 < nc; ++n1)
                    for (int n2 = 0; n2 < nc; ++n2) {
                        pr[n1 * nc + n2] = x1r[n1] * x2r[n2] - x1i[n1] * x2i[n2];
                        pi[n1 * nc + n2] = x1r[n1] * x2i[n2] + x1i[n1] * x2r[n2];
                        py[n1 * nc + n2] = y1[n1] * y2[n2];
                    }
                /* times the third corner, accumulated over triangles */
                for (int n12 = 0; n12 < nc * nc; ++n12) {
                    double sr = pr[n12], si = pi[n12], sy = py[n12];
                    double *orr = nr + (size_t)n12 * nc, *oi = ni + (size_t)n12 * nc;
                    double *od = dn + (size_t)n12 * nc;
                    for (int n3 = 0; n3 < nc; ++n3) {
                        orr[n3] += sr * x3r[n3] - si * x3i[n3];
                        oi[n3] += sr * x3i[n3] + si * x3r[n3];
                        od[n3] += sy * y3[n3];
                    }
                }
            }
        }
        tcount[t] = count;
        free(pr);
        free(pi);
        free(py);
    }
    free_rings(rc, nb);
    free(tr);
    free(ti);
    free(ty);
    return err ? -1 : 0;
}

/*
 * Closed-triangle counts for every ordered ring triple: T[(i*nb + j)*nb + l].
 * Cells with label -1 (unbinned or unoccupied) never take part.
 */
int orc_counts(int nt, int nb, const int *label, long long *T, int nthreads) {
    ring_cells *rc = build_rings(nt, nb, label);
    if (!rc) return -1;
    int ncell = nt * nt;
    size_t nb3 = (size_t)nb * nb * nb;
    memset(T, 0, nb3 * sizeof(long long));
    int *cu = (int *)malloc((size_t)ncell * sizeof(int));
    int *cv = (int *)malloc((size_t)ncell * sizeof(int));
    int *cl = (int *)malloc((size_t)ncell * sizeof(int));
    int n = 0;
    if (!cu || !cv || !cl) {
        free(cu);
        free(cv);
        free(cl);
        free_rings(rc, nb);
        return -1;
    }
    for (int c = 0; c < ncell; ++c)
        if (label[c] >= 0 && label[c] < nb) {
            cu[n] = c % nt - nt / 2;
            cv[n] = c / nt - nt / 2;
            cl[n] = label[c];
            ++n;
        }
    int err = 0;
#pragma omp parallel num_threads(nthreads_or_default(nthreads))
    {
        long long *loc = (long long *)calloc(nb3, sizeof(long long));
        if (!loc) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int p = 0; p < n; ++p) {
            if (!loc) continue;
            for (int q = 0; q < n; ++q) {
                int c3 = cell_of(nt, -cu[p] - cu[q], -cv[p] - cv[q]);
                if (c3 < 0) continue;
                int l = label[c3];
                if (l < 0 || l >= nb) continue;
                loc[((size_t)cl[p] * nb + cl[q]) * nb + l] += 1;
            }
        }
#pragma omp critical
        {
            if (loc)
                for (size_t k = 0; k < nb3; ++k) T[k] += loc[k];
        }
        free(loc);
    }
    free(cu);
    free(cv);
    free(cl);
    free_rings(rc, nb);
    return err ? -1 : 0;
}

/*
 * Single estimator points: pts[npts][6] = (i, j, l, nu1, nu2, nu3).
 * Outputs num_re/num_im/den[npts] and tcount[npts] (geometric count).
 * Parallel over the first corner of each point.
 */
int orc_points(int nt, int nc, int nb, const int *label, const double *xre,
               const double *xim, const double *y, int npts, const int *pts,
               double *num_re, double *num_im, double *den, long long *tcount,
               int nthreads) {
    int ncell = nt * nt;
    ring_cells *rc = build_rings(nt, nb, label);
    if (!rc) return -1;
    for (int s = 0; s < npts; ++s) {
        int ri = pts[6 * s], rj = pts[6 * s + 1], rl = pts[6 * s + 2];
        int n1 = pts[6 * s + 3], n2 = pts[6 * s + 4], n3 = pts[6 * s + 5];
        double ar = 0, ai = 0, ad = 0;
        long long cnt = 0;
        if (ri >= 0 && ri < nb && rj >= 0 && rj < nb && rl >= 0 && rl < nb && n1 >= 0 &&
            n1 < nc && n2 >= 0 && n2 < nc && n3 >= 0 && n3 < nc) {
            const ring_cells *a = &rc[ri], *b = &rc[rj];
            const double *x1r = xre + (size_t)n1 * ncell, *x1i = xim + (size_t)n1 * ncell;
            const double *x2r = xre + (size_t)n2 * ncell, *x2i = xim + (size_t)n2 * ncell;
            const double *x3r = xre + (size_t)n3 * ncell, *x3i = xim + (size_t)n3 * ncell;
            const double *y1 = y + (size_t)n1 * ncell, *y2 = y + (size_t)n2 * ncell;
            const double *y3 = y + (size_t)n3 * ncell;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : ar, ai, ad, cnt) \
    num_threads(nthreads_or_default(nthreads))
            for (int p = 0; p < a->n; ++p) {
                int c1 = a->cell[p];
                for (int q = 0; q < b->n; ++q) {
                    int c3 = cell_of(nt, -a->u[p] - b->u[q], -a->v[p] - b->v[q]);
                    if (c3 < 0 || label[c3] != rl) continue;
                    int c2 = b->cell[q];
                    double sr = x1r[c1] * x2r[c2] - x1i[c1] * x2i[c2];
                    double si = x1r[c1] * x2i[c2] + x1i[c1] * x2r[c2];
                    ar += sr * x3r[c3] - si * x3i[c3];
                    ai += sr * x3i[c3] + si * x3r[c3];
                    ad += y1[c1] * y2[c2] * y3[c3];
                    ++cnt;
                }
            }
        }
        num_re[s] = ar;
        num_im[s] = ai;
        den[s] = ad;
        tcount[s] = cnt;
    }
    free_rings(rc, nb);
    return 0;
}

/*
 * Collapsed-plane points for one channel window [nu_lo, nu_hi):
 * pts[npts][5] = (i, j, l, d1, d2).  For every nu3 in the window with
 * nu3 + d1 and nu3 + d2 also in the window, the per-triple numerator and
 * denominator are accumulated over triangles into per-nu3 arrays; then
 *   ratio_sum[s] = sum over nu3 with den > 0 of num/den  (real and imaginary)
 *   nvalid[s]    = number of such nu3.
 * The Section 3.2 collapse takes the mean ratio_sum / nvalid.
 */
int orc_delta_points_block(int nt, int nc, int nb, const int *label, const double *xre,
                           const double *xim, const double *y, const int *blk, int npts,
                           const int *pts, double *ratio_re, double *ratio_im,
                           long long *nvalid, int nthreads) {
    int ncell = nt * nt;
    for (int k = 0; k < 3; ++k)
        if (blk[2 * k] < 0 || blk[2 * k + 1] > nc || blk[2 * k] >= blk[2 * k + 1]) return -2;
    int nu_lo = blk[4], nu_hi = blk[5];
    ring_cells *rc = build_rings(nt, nb, label);
    double *tr = transpose_cc(xre, nc, ncell);
    double *ti = transpose_cc(xim, nc, ncell);
    double *ty = transpose_cc(y, nc, ncell);
    if (!rc || !tr || !ti || !ty) {
        free_rings(rc, nb);
        free(tr);
        free(ti);
        free(ty);
        return -1;
    }
    int nth = nthreads_or_default(nthreads);
    int nw = nu_hi - nu_lo;
    int err = 0;
    double *acc = (double *)calloc((size_t)nth * 3 * nw, sizeof(double));
    if (!acc) err = 1;
    for (int s = 0; s < npts && !err; ++s) {
        int ri = pts[5 * s], rj = pts[5 * s + 1], rl = pts[5 * s + 2];
        int d1 = pts[5 * s + 3], d2 = pts[5 * s + 4];
        memset(acc, 0, (size_t)nth * 3 * nw * sizeof(double));
        /* window channels nu3 such that all three channels stay inside their ranges */
        int lo = nu_lo, hi = nu_hi;
        if (blk[0] - d1 > lo) lo = blk[0] - d1;
        if (blk[2] - d2 > lo) lo = blk[2] - d2;
        if (blk[1] - d1 < hi) hi = blk[1] - d1;
        if (blk[3] - d2 < hi) hi = blk[3] - d2;
        if (ri >= 0 && ri < nb && rj >= 0 && rj < nb && rl >= 0 && rl < nb && lo < hi) {
            const ring_cells *a = &rc[ri], *b = &rc[rj];
#pragma omp parallel num_threads(nth)
            {
                int tid = 0;
#ifdef _OPENMP
                tid = omp_get_thread_num();
#endif
                double *ar = acc + (size_t)tid * 3 * nw, *ai = ar + nw, *ad = ai + nw;
#pragma omp for schedule(dynamic, 8)
                for (int p = 0; p < a->n; ++p) {
                    for (int q = 0; q < b->n; ++q) {
                        int c3 = cell_of(nt, -a->u[p] - b->u[q], -a->v[p] - b->v[q]);
                        if (c3 < 0 || label[c3] != rl) continue;
                        const double *x1r = tr + (size_t)a->cell[p] * nc, *x1i = ti + (size_t)a->cell[p] * nc;
                        const double *x2r = tr + (size_t)b->cell[q] * nc, *x2i = ti + (size_t)b->cell[q] * nc;
                        const double *x3r = tr + (size_t)c3 * nc, *x3i = ti + (size_t)c3 * nc;
                        const double *y1 = ty + (size_t)a->cell[p] * nc, *y2 = ty + (size_t)b->cell[q] * nc;
                        const double *y3 = ty + (size_t)c3 * nc;
                        for (int n3 = lo; n3 < hi; ++n3) {
                            int n1 = n3 + d1, n2 = n3 + d2;
                            double sr = x1r[n1] * x2r[n2] - x1i[n1] * x2i[n2];
                            double si = x1r[n1] * x2i[n2] + x1i[n1] * x2r[n2];
                            ar[n3 - nu_lo] += sr * x3r[n3] - si * x3i[n3];
                            ai[n3 - nu_lo] += sr * x3i[n3] + si * x3r[n3];
                            ad[n3 - nu_lo] += y1[n1] * y2[n2] * y3[n3];
                        }
                    }
                }
            }
        }
        double sr = 0, si = 0;
        long long nv = 0;
        for (int n3 = lo; n3 < hi; ++n3) {
            double nr = 0, niv = 0, dd = 0;
            for (int t = 0; t < nth; ++t) {
                const double *ar = acc + (size_t)t * 3 * nw;
                nr += ar[n3 - nu_lo];
                niv += ar[nw + n3 - nu_lo];
                dd += ar[2 * nw + n3 - nu_lo];
            }
            if (dd > 0) {
                sr += nr / dd;
                si += niv / dd;
                ++nv;
            }
        }
        ratio_re[s] = sr;
        ratio_im[s] = si;
        nvalid[s] = nv;
    }
    free(acc);
    free_rings(rc, nb);
    free(tr);
    free(ti);
    free(ty);
    return err ? -1 : 0;
}

/* Cube window [nu_lo, nu_hi) for all three channels. */
int orc_delta_points(int nt, int nc, int nb, const int *label, const double *xre,
                     const double *xim, const double *y, int nu_lo, int nu_hi, int npts,
                     const int *pts, double *ratio_re, double *ratio_im, long long *nvalid,
                     int nthreads) {
    const int blk[6] = {nu_lo, nu_hi, nu_lo, nu_hi, nu_lo, nu_hi};
    return orc_delta_points_block(nt, nc, nb, label, xre, xim, y, blk, npts, pts, ratio_re,
                                  ratio_im, nvalid, nthreads);
}
