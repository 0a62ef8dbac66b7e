/*
 * packer.c -- geometric packing of spheres for the seeded input generator.
 *
 * Overlap removal by Gauss-Seidel sweeps over a cell list: every overlapping
 * pair is pushed apart along its centre line by half the overlap until the
 * largest overlap is below tol * (mean radius).  Pure geometry: no contact
 * law, no dynamics.  Periodic cube (kind 0) or cylindrical annulus (kind 1:
 * r_out + R <= r <= Rc - R, or r <= Rc - R without a cavity (r_out = 0),
 * z >= R, free top surface).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static double wrapd(double a, double L) {
    a = fmod(a, L);
    if (a < 0) a += L;
    if (a >= L) a -= L;
    return a;
}

static void constrain(int kind, double* p, double R, const double* geo) {
    if (kind == 0) {
        for (int k = 0; k < 3; ++k) p[k] = wrapd(p[k], geo[0]);
        return;
    }
    double Rc = geo[0], r_out = geo[1], h_bed = geo[2];
    double r = sqrt(p[0] * p[0] + p[1] * p[1]);
    double rmin = r_out > 0.0 ? r_out + R : 0.0, rmax = Rc - R; /* r_out = 0: no cavity */
    if (rmax < rmin) rmax = rmin;
    double t = r < rmin ? rmin : (r > rmax ? rmax : r);
    if (r > 0) {
        p[0] *= t / r;
        p[1] *= t / r;
    } else {
        p[0] = t;
    }
    /* the bed top is free: spheres may rise above h_bed while overlaps resolve */
    (void)h_bed;
    if (p[2] < R) p[2] = R;
}

/* geo: kind 0 -> {L}; kind 1 -> {Rc, r_out, h_bed}.  Returns sweeps used
 * (negative if not converged). */
int gen_pack(int64_t n, double* x, const double* R, int kind, const double* geo, int iters,
             double tol) {
    if (n <= 0) return 0;
    double Rmax = 0, Rsum = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (R[i] > Rmax) Rmax = R[i];
        Rsum += R[i];
    }
    double Rmean = Rsum / (double)n;
    double lo[3], ext[3];
    if (kind == 0) {
        for (int k = 0; k < 3; ++k) { lo[k] = 0; ext[k] = geo[0]; }
    } else {
        lo[0] = lo[1] = -geo[0];
        ext[0] = ext[1] = 2 * geo[0];
        lo[2] = 0;
        ext[2] = geo[2] > 0 ? 1.5 * geo[2] : 1e-9;
    }
    double h = 2.0 * Rmean;
    int nc[3];
    for (;;) {
        double tot = 1;
        for (int k = 0; k < 3; ++k) {
            nc[k] = (int)floor(ext[k] / h);
            if (nc[k] < 1) nc[k] = 1;
            tot *= nc[k];
        }
        if (tot <= 4.0e7) break;
        h *= 1.25;
    }
    double hc[3];
    for (int k = 0; k < 3; ++k) hc[k] = ext[k] / nc[k];
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (ncell + 1));
    int64_t* items = (int64_t*)malloc(sizeof(int64_t) * n);
    int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * n);
    int used = -iters;
    for (int64_t i = 0; i < n; ++i) constrain(kind, &x[3 * i], R[i], geo);
    for (int it = 0; it < iters; ++it) {
        for (int64_t c = 0; c <= ncell; ++c) start[c] = 0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t ci[3];
            for (int k = 0; k < 3; ++k) {
                int64_t t = (int64_t)floor((x[3 * i + k] - lo[k]) / hc[k]);
                if (t < 0) t = 0;
                if (t >= nc[k]) t = nc[k] - 1;
                ci[k] = t;
            }
            cell[i] = (ci[2] * nc[1] + ci[1]) * nc[0] + ci[0];
            start[cell[i] + 1]++;
        }
        for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
        for (int64_t i = 0; i < n; ++i) items[start[cell[i]]++] = i;
        for (int64_t c = ncell; c > 0; --c) start[c] = start[c - 1];
        start[0] = 0;
        double worst = 0;
        for (int64_t qi = 0; qi < n; ++qi) {
            int64_t i = items[qi];
            int64_t c = cell[i];
            int ci[3] = {(int)(c % nc[0]), (int)((c / nc[0]) % nc[1]), (int)(c / ((int64_t)nc[0] * nc[1]))};
            int lst[3][64], cnt[3];
            for (int k = 0; k < 3; ++k) {
                int r = (int)ceil((2.0 * R[i]) / hc[k]);
                cnt[k] = 0;
                if (kind == 0 && 2 * r + 1 >= nc[k]) {
                    for (int a = 0; a < nc[k] && a < 64; ++a) lst[k][cnt[k]++] = a;
                } else {
                    for (int a = ci[k] - r; a <= ci[k] + r && cnt[k] < 64; ++a) {
                        int b = a;
                        if (kind == 0) b = ((a % nc[k]) + nc[k]) % nc[k];
                        else if (a < 0 || a >= nc[k]) continue;
                        lst[k][cnt[k]++] = b;
                    }
                }
            }
            for (int az = 0; az < cnt[2]; ++az)
                for (int ay = 0; ay < cnt[1]; ++ay)
                    for (int ax = 0; ax < cnt[0]; ++ax) {
                        int64_t c2 = ((int64_t)lst[2][az] * nc[1] + lst[1][ay]) * nc[0] + lst[0][ax];
                        for (int64_t q = start[c2]; q < start[c2 + 1]; ++q) {
                            int64_t j = items[q];
                            if (j == i) continue;
                            if (R[j] > R[i] || (R[j] == R[i] && j < i)) continue;
                            double d[3];
                            for (int k = 0; k < 3; ++k) {
                                d[k] = x[3 * j + k] - x[3 * i + k];
                                if (kind == 0) {
                                    double L = geo[0];
                                    if (d[k] > 0.5 * L) d[k] -= L;
                                    else if (d[k] < -0.5 * L) d[k] += L;
                                }
                            }
                            double S = R[i] + R[j];
                            double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                            if (d2 >= S * S) continue;
                            double dist = sqrt(d2);
                            double ov = S - dist;
                            if (ov > worst) worst = ov;
                            double u[3];
                            if (dist > 0) {
                                for (int k = 0; k < 3; ++k) u[k] = d[k] / dist;
                            } else {
                                u[0] = 1; u[1] = 0; u[2] = 0;
                            }
                            for (int k = 0; k < 3; ++k) {
                                x[3 * i + k] -= 0.5 * ov * u[k];
                                x[3 * j + k] += 0.5 * ov * u[k];
                            }
                            constrain(kind, &x[3 * j], R[j], geo);
                        }
                    }
            constrain(kind, &x[3 * i], R[i], geo);
        }
        if (worst < tol * Rmean) {
            used = it + 1;
            break;
        }
    }
    free(start);
    free(items);
    free(cell);
    return used;
}
