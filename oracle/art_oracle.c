/*
 * art_oracle.c -- plain, slow, FP64 CPU oracle for adaptive ray tracing (ART) of point
 * sources through a uniform Cartesian grid, following Kim, Kim, Ostriker & Skinner (2017),
 * Sec. 2.1 (Eqs. e:RT2, e:Erad, e:Frad and the splitting / termination rules), Sec. 2.3
 * (Eq. e:photrate2 and the ionizing opacity chi_i = n_HI sigma_H + n_H sigma_d), and the
 * HEALPix nested scheme of Gorski et al. (2005, ApJ 622, 759) cited in Sec. 2.1.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the independent reference that the CUDA path is
 * checked against; it shares no code with it. Only the test suite, the package smoke check
 * and the bench's CPU-baseline leg may load it. The library never calls it.
 *
 * Conventions (code units c = 1, h nu_i = 1):
 *   - grid: nx*ny*nz cells of side dx starting at lo[3]; flat index i + nx*(j + ny*k);
 *   - positions are converted to cell units u = (x - lo)/dx, and all path lengths are
 *     handled in cell units and multiplied by dx when an optical depth or deposit is formed;
 *   - per cell the oracle accumulates G = sum L_in ds phi(dtau) (which equals sum dL/chi,
 *     finite as chi -> 0) and F = sum dL n; then Gamma = sigma_H G / dV (Eq. e:photrate2
 *     divided by n_HI), E = G / dV (Eq. e:Erad) and f_rad = F / dV (chi F / c with
 *     Eq. e:Frad).
 * Readings of points the paper leaves open (each listed in the design notes):
 *   - split at exactly r = r_max(l); children start at x_src + r_max(l) n_child, inherit
 *     tau and carry L/4 each (Sec. 2.1);
 *   - l_max per source: smallest l >= l0 with r_max(l) >= distance to the farthest box
 *     corner, capped at 13, unless a fixed cap is given; rays at l_max never split;
 *   - termination when tau > tau_max after a segment (the segment's deposit is kept), or
 *     when the ray leaves the box;
 *   - start cell: floor of the position; on a face with n_a < 0 the lower cell; a zero
 *     component keeps floor;
 *   - axes whose face crossings agree to 1e-12 relative step together; segments of zero
 *     length are neither deposited nor counted;
 *   - directions: phi/pi is formed as an exact rational and reduced with integer
 *     arithmetic, so components are exactly 0 or +-1 where they should be, cos = sin at
 *     pi/4; after rotation any component below 2^-24 in magnitude is set to 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_LEVEL 13
#define OR_NLEVELS 20
#define OR_TIE_REL 1e-12
#define OR_NEAR 1e-5

/* ------------------------------------------------------------------------------------- */
/* HEALPix nested scheme (Gorski et al. 2005, Sec. 4-5)                                   */
/* ------------------------------------------------------------------------------------- */

static void or_split_bits(uint64_t q, int64_t* ix, int64_t* iy)
{
    int64_t x = 0, y = 0;
    for (int b = 0; b < 31; ++b) {
        x |= (int64_t)((q >> (2 * b)) & 1u) << b;
        y |= (int64_t)((q >> (2 * b + 1)) & 1u) << b;
    }
    *ix = x;
    *iy = y;
}

static uint64_t or_merge_bits(int64_t ix, int64_t iy)
{
    uint64_t q = 0;
    for (int b = 0; b < 31; ++b) {
        q |= (uint64_t)((ix >> b) & 1) << (2 * b);
        q |= (uint64_t)((iy >> b) & 1) << (2 * b + 1);
    }
    return q;
}

/* sin and cos of pi*a/b for integers a, b > 0: exact at multiples of 1/2, equal at 1/4. */
static void or_sincospi_ratio(int64_t a, int64_t b, double* s, double* c)
{
    int64_t per = 2 * b;
    a %= per;
    if (a < 0) a += per;
    double ss = 1.0, sc = 1.0;
    if (a >= b) { a -= b; ss = -1.0; sc = -1.0; }   /* angle - pi */
    if (2 * a > b) { a = b - a; sc = -sc; }          /* pi - angle */
    double sv, cv;
    if (a == 0) { sv = 0.0; cv = 1.0; }
    else if (2 * a == b) { sv = 1.0; cv = 0.0; }
    else if (4 * a == b) { sv = sqrt(0.5); cv = sv; }
    else { double x = M_PI * (double)a / (double)b; sv = sin(x); cv = cos(x); }
    *s = ss * sv;
    *c = sc * cv;
}

/* Unit vector of the centre of nested pixel pix at level l (N_side = 2^l). */
void or_pix2vec(int level, uint64_t pix, double v[3])
{
    static const int ring_row[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
    static const int ring_col[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};
    const int64_t ns = (int64_t)1 << level;
    const uint64_t per_face = (uint64_t)ns * (uint64_t)ns;
    const int face = (int)(pix / per_face);
    int64_t ix, iy;
    or_split_bits(pix % per_face, &ix, &iy);
    const int64_t jr = (int64_t)ring_row[face] * ns - ix - iy - 1; /* ring index 1..4ns-1 */
    int64_t nr;
    int shift;
    double z, sth;
    if (jr < ns) {                 /* north polar cap */
        nr = jr; shift = 0;
        double a = (double)(nr * nr) / (3.0 * (double)ns * (double)ns);
        z = 1.0 - a; sth = sqrt(a * (2.0 - a));
    } else if (jr > 3 * ns) {      /* south polar cap */
        nr = 4 * ns - jr; shift = 0;
        double a = (double)(nr * nr) / (3.0 * (double)ns * (double)ns);
        z = a - 1.0; sth = sqrt(a * (2.0 - a));
    } else {                       /* equatorial belt */
        nr = ns; shift = (int)((jr - ns) & 1);
        z = (double)(2 * (2 * ns - jr)) / (3.0 * (double)ns);
        sth = sqrt((1.0 - z) * (1.0 + z));
    }
    int64_t jp = ((int64_t)ring_col[face] * nr + ix - iy + 1 + shift) / 2;
    if (jp > 4 * nr) jp -= 4 * nr;
    if (jp < 1) jp += 4 * nr;
    double s, c;
    or_sincospi_ratio(2 * jp - shift - 1, 4 * nr, &s, &c); /* phi/pi = (2jp-shift-1)/(4nr) */
    v[0] = sth * c;
    v[1] = sth * s;
    v[2] = z;
}

/* Nested pixel containing direction v at level l (used by the tests as an independent
 * inverse of or_pix2vec). */
uint64_t or_vec2pix(int level, const double v[3])
{
    const int64_t ns = (int64_t)1 << level;
    double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double z = v[2] / r;
    double phi = atan2(v[1], v[0]);
    if (phi < 0) phi += 2.0 * M_PI;
    double tt = phi / (0.5 * M_PI);
    if (tt >= 4.0) tt -= 4.0;
    double za = fabs(z);
    int face;
    int64_t ix, iy;
    if (za <= 2.0 / 3.0) {
        double t1 = (double)ns * (0.5 + tt);
        double t2 = (double)ns * (0.75 * z);
        int64_t jp = (int64_t)floor(t1 - t2); /* ascending edge line index */
        int64_t jm = (int64_t)floor(t1 + t2); /* descending edge line index */
        int64_t fp = jp / ns, fm = jm / ns;
        if (fp == fm) face = (int)((fp % 4) + 4);
        else if (fp < fm) face = (int)(fp % 4);
        else face = (int)((fm % 4) + 8);
        ix = jm & (ns - 1);
        iy = ns - (jp & (ns - 1)) - 1;
    } else {
        int ntt = (int)tt;
        if (ntt > 3) ntt = 3;
        double tp = tt - ntt;
        double tmp = (double)ns * sqrt(3.0 * (1.0 - za));
        int64_t jp = (int64_t)(tp * tmp);
        int64_t jm = (int64_t)((1.0 - tp) * tmp);
        if (jp > ns - 1) jp = ns - 1;
        if (jm > ns - 1) jm = ns - 1;
        if (z >= 0) { face = ntt; ix = ns - jm - 1; iy = ns - jp - 1; }
        else { face = ntt + 8; ix = jp; iy = jm; }
    }
    return (uint64_t)face * (uint64_t)ns * (uint64_t)ns + or_merge_bits(ix, iy);
}

/* ------------------------------------------------------------------------------------- */
/* Problem description                                                                    */
/* ------------------------------------------------------------------------------------- */

typedef struct {
    int n[3];
    double dx;
    const float* nH0;   /* neutral hydrogen density per cell */
    const float* nH;    /* total hydrogen density per cell (dust), may be NULL */
    double sigma_H, sigma_d;
    int level0;
    int level_cap;      /* < 0: automatic per source */
    double m_ray, tau_max;
    double rot[9];
    int use_rot;
    int two_bin;        /* a second, non-ionizing bin attenuated by dust only (Sec. 2.3) */
    double rmax_unit;   /* sqrt(3/(pi m_ray)): r_max(l) = rmax_unit * 2^l (cells) */
    double dmax;        /* rays end at this distance from their source (cells); INFINITY: none */
    long long* hits;    /* deposits per cell (counted when not NULL; test bookkeeping only) */
} or_problem;

typedef struct {
    long long crossings, rays, near_tie_rays;
    long long per_level[OR_NLEVELS];
    long long destroy;  /* sum of 4^(lmax_global - l) over retired rays */
    int level_reached;
    double absorbed, escaped, dropped;
    double absorbed_n, escaped_n, dropped_n;  /* non-ionizing bin (two-bin traces) */
} or_tally;

typedef struct {
    int level;
    uint64_t pix;
    double L, tau;
    double Ln, taun;  /* non-ionizing bin (two-bin traces), else 0 */
} or_ray;

static double or_rmax(const or_problem* P, int level)
{
    return P->rmax_unit * ldexp(1.0, level);
}

static void or_direction(const or_problem* P, int level, uint64_t pix, double n[3])
{
    double v[3];
    or_pix2vec(level, pix, v);
    if (P->use_rot) {
        for (int a = 0; a < 3; ++a)
            n[a] = P->rot[3 * a + 0] * v[0] + P->rot[3 * a + 1] * v[1] + P->rot[3 * a + 2] * v[2];
    } else {
        n[0] = v[0]; n[1] = v[1]; n[2] = v[2];
    }
    for (int a = 0; a < 3; ++a)
        if (fabs(n[a]) < 0x1p-24) n[a] = 0.0;
}

/* l_max for a source at u (cell units): smallest l >= l0 whose r_max reaches the farthest
 * box corner, capped at 13, or the fixed cap when one is given. */
static int or_level_max(const or_problem* P, const double u[3])
{
    if (P->level_cap >= 0) return P->level_cap;
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = fmax(u[a], (double)P->n[a] - u[a]);
        d2 += e * e;
    }
    double rfar = sqrt(d2);
    int l = P->level0;
    while (l < OR_MAX_LEVEL && or_rmax(P, l) < rfar) ++l;
    return l;
}

static double or_phi(double x)  /* (1 - e^-x)/x, phi(0) = 1 */
{
    if (x < 1e-4) return 1.0 - 0.5 * x + x * x / 6.0;
    return -expm1(-x) / x;
}

static double or_dphi(double x) /* d phi / dx = (e^-x (1 + x) - 1)/x^2 */
{
    if (x < 1e-3) return -0.5 + x / 3.0 - x * x / 8.0;
    return (exp(-x) * (1.0 + x) - 1.0) / (x * x);
}

/* One segment of a ray inside a cell: everything later steps need. */
typedef struct {
    int64_t cell;
    double ds;     /* physical length */
    double dtau, dtauH;
    double Lin;
} or_seg;

typedef struct {
    or_seg* v;
    size_t n, cap;
} or_segvec;

static void or_segvec_push(or_segvec* s, or_seg g)
{
    if (s->n == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 256;
        s->v = (or_seg*)realloc(s->v, s->cap * sizeof(or_seg));
    }
    s->v[s->n++] = g;
}

enum { OR_END_EXIT = 0, OR_END_DROP = 1, OR_END_SPLIT = 2 };

/*
 * Walk one ray (level, pixel, L, tau) from r_start to its end: the box exit, tau > tau_max,
 * r_max(level) when level < lmax (Sec. 2.1), or the cutoff distance d_max from the source
 * (the terminated rays of the weak-scaling test, Sec. 3.1; reported like an exit). Face crossings are measured from the source
 * (t_a = (face_a - u_a)/n_a, never incremented), so no drift builds up. Calls deposit per
 * segment when acc != NULL, records segments when segs != NULL. Returns the end reason;
 * the ray's L and tau are updated to their values at the end.
 */
static void or_add(double* p, double v, int atomic)
{
    if (atomic) {
#pragma omp atomic
        *p += v;
    } else {
        *p += v;
    }
}

static int or_walk(const or_problem* P, const double u[3], or_ray* ray, int lmax,
                   double* acc, int64_t ncell, int atomic, or_segvec* segs, or_tally* T,
                   int* near)
{
    double n[3];
    or_direction(P, ray->level, ray->pix, n);
    const double r0 = ray->level > P->level0 ? or_rmax(P, ray->level - 1) : 0.0;
    /* the walk ends at the split radius (levels below lmax) or at d_max, whichever comes
     * first; at equal radii the cut wins (the ray is not split) */
    const double rsplit = ray->level < lmax ? or_rmax(P, ray->level) : INFINITY;
    const double rend = fmin(rsplit, P->dmax);
    const int cut = P->dmax <= rsplit;

    int64_t c[3];
    double tn[3], dt[3];
    int step[3];
    for (int a = 0; a < 3; ++a) {
        double p = u[a] + r0 * n[a];
        double f = floor(p);
        c[a] = (int64_t)f;
        if (n[a] < 0.0 && p == f) c[a] -= 1;
        if (r0 > 0.0 && n[a] != 0.0 && fabs(p - floor(p + 0.5)) < OR_NEAR) *near = 1;
        if (n[a] > 0.0) { step[a] = 1; tn[a] = ((double)(c[a] + 1) - u[a]) / n[a]; dt[a] = 1.0 / n[a]; }
        else if (n[a] < 0.0) { step[a] = -1; tn[a] = ((double)c[a] - u[a]) / n[a]; dt[a] = -1.0 / n[a]; }
        else { step[a] = 0; tn[a] = INFINITY; dt[a] = INFINITY; }
    }
    for (int a = 0; a < 3; ++a)
        if (c[a] < 0 || c[a] >= P->n[a]) return OR_END_EXIT;

    const double dx = P->dx;
    double t = r0;
    for (;;) {
        double tmin = fmin(tn[0], fmin(tn[1], tn[2]));
        double tend = fmin(tmin, rend);
        double ds = tend - t;
        if (ds > 0.0) {
            int64_t idx = c[0] + (int64_t)P->n[0] * (c[1] + (int64_t)P->n[1] * c[2]);
            double chiH = (double)P->nH0[idx] * P->sigma_H;
            double chi = chiH + (P->nH ? (double)P->nH[idx] * P->sigma_d : 0.0);
            double dsp = ds * dx;
            double dtau = chi * dsp;
            double dL = -ray->L * expm1(-dtau);
            /* non-ionizing bin: chi_n = n_H sigma_d; its momentum adds to the force
             * (Eq. e:radforce sums chi_nu F_nu / c over the bins) */
            double dtaun = 0.0, dLn = 0.0;
            if (P->two_bin) {
                dtaun = (P->nH ? (double)P->nH[idx] * P->sigma_d : 0.0) * dsp;
                dLn = -ray->Ln * expm1(-dtaun);
            }
            if (acc) {
                double G = ray->L * dsp * or_phi(dtau);
                or_add(acc + idx, G, atomic);
                or_add(acc + ncell + idx, (dL + dLn) * n[0], atomic);
                or_add(acc + 2 * ncell + idx, (dL + dLn) * n[1], atomic);
                or_add(acc + 3 * ncell + idx, (dL + dLn) * n[2], atomic);
                if (P->hits) {
#pragma omp atomic
                    P->hits[idx] += 1;
                }
            }
            if (segs) {
                or_seg g = {idx, dsp, dtau, chiH * dsp, ray->L};
                or_segvec_push(segs, g);
            }
            if (ds < OR_NEAR) *near = 1;
            ray->L -= dL;
            ray->tau += dtau;
            ray->Ln -= dLn;
            ray->taun += dtaun;
            T->crossings += 1;
            T->absorbed += dL;
            T->absorbed_n += dLn;
            /* the packet is used up once every bin it carries is: with two bins the
             * dust-only depth (never larger than the ionizing one) decides */
            const double tau_end = P->two_bin ? ray->taun : ray->tau;
            if (fabs(tau_end - P->tau_max) < 1e-4 * P->tau_max) *near = 1;
            if (tau_end > P->tau_max) return OR_END_DROP;
        }
        if (rend <= tmin) {
            if (tmin - rend < OR_NEAR) *near = 1;
            return cut ? OR_END_EXIT : OR_END_SPLIT;
        }
        if (tmin - rend > -OR_NEAR && rend < INFINITY) *near = 1;
        /* step every axis whose crossing ties with the earliest one */
        double tol = OR_TIE_REL * tmin;
        int out = 0;
        for (int a = 0; a < 3; ++a) {
            if (step[a] != 0 && tn[a] - tmin <= tol) {
                c[a] += step[a];
                tn[a] = ((double)(step[a] > 0 ? c[a] + 1 : c[a]) - u[a]) / n[a];
                if (c[a] < 0 || c[a] >= P->n[a]) out = 1;
            } else if (step[a] != 0 && tn[a] - tmin < OR_NEAR) {
                *near = 1;
            }
        }
        (void)dt;
        if (out) return OR_END_EXIT;
        t = tend;
    }
}

/* Depth-first (last-in first-out) trace of one base ray and all its descendants, as in
 * Sec. 2.2 where children are stacked on top of their parent. */
static void or_trace_tree(const or_problem* P, const double u[3], int lmax, int lmax_glob,
                          or_ray root, double* acc, int64_t ncell, int atomic, or_tally* T)
{
    or_ray stack[4 * OR_NLEVELS + 8];
    int top = 0;
    stack[top++] = root;
    while (top > 0) {
        or_ray ray = stack[--top];
        int near = 0;
        T->rays += 1;
        T->per_level[ray.level] += 1;
        if (ray.level > T->level_reached) T->level_reached = ray.level;
        int end = or_walk(P, u, &ray, lmax, acc, ncell, atomic, NULL, T, &near);
        if (near) T->near_tie_rays += 1;
        if (end == OR_END_SPLIT) {
            for (int k = 3; k >= 0; --k) {
                or_ray ch = {ray.level + 1, 4 * ray.pix + (uint64_t)k, 0.25 * ray.L, ray.tau,
                             0.25 * ray.Ln, ray.taun};
                stack[top++] = ch;
            }
        } else {
            if (end == OR_END_EXIT) { T->escaped += ray.L; T->escaped_n += ray.Ln; }
            else { T->dropped += ray.L; T->dropped_n += ray.Ln; }
            T->destroy += (long long)1 << (2 * (lmax_glob - ray.level));
        }
    }
}

static int or_setup(or_problem* P, int nx, int ny, int nz, double dx, const float* nH0,
                    const float* nH, int level0, int level_cap, double m_ray, double tau_max,
                    double sigma_H, double sigma_d, const double* rot, double d_max)
{
    if (nx <= 0 || ny <= 0 || nz <= 0 || !(dx > 0) || !nH0) return -1;
    if (d_max != d_max) return -1;
    if (level0 < 0 || level0 > 12 || !(m_ray > 0) || !(tau_max > 0)) return -1;
    if (level_cap >= 0 && (level_cap < level0 || level_cap > OR_MAX_LEVEL)) return -1;
    P->n[0] = nx; P->n[1] = ny; P->n[2] = nz;
    P->dx = dx; P->nH0 = nH0; P->nH = nH;
    P->sigma_H = sigma_H; P->sigma_d = sigma_d;
    P->level0 = level0; P->level_cap = level_cap;
    P->m_ray = m_ray; P->tau_max = tau_max;
    P->use_rot = rot != NULL;
    P->two_bin = 0;
    for (int i = 0; i < 9; ++i) P->rot[i] = rot ? rot[i] : (i % 4 == 0 ? 1.0 : 0.0);
    P->rmax_unit = sqrt(3.0 / (M_PI * m_ray));
    P->dmax = d_max > 0.0 ? d_max / dx : INFINITY;
    P->hits = NULL;
    return 0;
}

static int or_source_cells(const or_problem* P, int nsrc, const double* lo, const double* pos,
                           double* u)
{
    for (int s = 0; s < nsrc; ++s)
        for (int a = 0; a < 3; ++a) {
            u[3 * s + a] = (pos[3 * s + a] - lo[a]) / P->dx;
            if (!(u[3 * s + a] > 0.0 && u[3 * s + a] < (double)P->n[a])) return -1;
        }
    return 0;
}

/*
 * Full multi-source trace. acc: 4*ncell doubles (G, Fx, Fy, Fz blocks), overwritten.
 * pix_stride >= 1: trace only the base rays whose pixel index is a multiple of pix_stride
 * (with all their descendants), a bounded sample for timing; 1 traces everything.
 * hits: ncell counts of deposits per cell (overwritten), or NULL.
 * Ln: per-source non-ionizing luminosity (a second bin, attenuated by n_H sigma_d), or NULL
 * for one bin. dstat[8] = {L_in, absorbed, escaped, dropped} of the ionizing bin, then the
 * same four of the non-ionizing bin.
 * istat[8 + OR_NLEVELS] = {crossings, rays, near_tie_rays, destroy, destroy_expected,
 *                          level_reached, lmax_global, 0, per_level[0..19]}.
 * Returns 0, or -1 on invalid input.
 */
int or_trace(int nx, int ny, int nz, const double* lo, double dx, const float* nH0,
             const float* nH, int nsrc, const double* pos, const double* L, const double* Ln,
             int level0,
             int level_cap, double m_ray, double tau_max, double sigma_H, double sigma_d,
             const double* rot, double d_max, double* acc, double* dstat, long long* istat,
             int nthreads, int pix_stride, long long* hits)
{
    or_problem P;
    if (or_setup(&P, nx, ny, nz, dx, nH0, nH, level0, level_cap, m_ray, tau_max, sigma_H,
                 sigma_d, rot, d_max))
        return -1;
    if (nsrc < 0 || pix_stride < 1) return -1;
    P.hits = hits;
    P.two_bin = Ln != NULL;
    double* u = (double*)malloc(sizeof(double) * 3 * (size_t)(nsrc > 0 ? nsrc : 1));
    if (or_source_cells(&P, nsrc, lo, pos, u)) { free(u); return -1; }
    const int64_t ncell = (int64_t)nx * ny * nz;
    memset(acc, 0, sizeof(double) * 4 * (size_t)ncell);
    if (hits) memset(hits, 0, sizeof(long long) * (size_t)ncell);
    double Ln_in = 0.0;
    for (int s = 0; s < nsrc && Ln; ++s) Ln_in += Ln[s];
    int lmax_glob = level0;
    double Lin = 0.0;
    for (int s = 0; s < nsrc; ++s) {
        int lm = or_level_max(&P, u + 3 * s);
        if (lm > lmax_glob) lmax_glob = lm;
        Lin += L[s];
    }
    const long long nbase = 12LL << (2 * level0);
    const long long nwork = (long long)nsrc * nbase;
    or_tally tot;
    memset(&tot, 0, sizeof(tot));
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        or_tally T;
        memset(&T, 0, sizeof(T));
        double* myacc = acc;
        int nt = 1;
#ifdef _OPENMP
        nt = omp_get_num_threads();
#endif
        /* private accumulators while they stay small, shared atomics beyond 1 GiB */
        const int atomic = nt > 1 && (double)nt * 32.0 * (double)ncell > 1073741824.0;
        if (nt > 1 && !atomic) myacc = (double*)calloc(4 * (size_t)ncell, sizeof(double));
#pragma omp for schedule(dynamic, 16)
        for (long long w = 0; w < nwork; ++w) {
            int s = (int)(w / nbase);
            uint64_t p = (uint64_t)(w % nbase);
            if (p % (uint64_t)pix_stride != 0) continue;
            int lm = or_level_max(&P, u + 3 * s);
            or_ray root = {level0, p, L[s] / (double)nbase, 0.0,
                           Ln ? Ln[s] / (double)nbase : 0.0, 0.0};
            or_trace_tree(&P, u + 3 * s, lm, lmax_glob, root, myacc, ncell, atomic, &T);
        }
#pragma omp critical
        {
            if (myacc != acc) {
                for (int64_t i = 0; i < 4 * ncell; ++i) acc[i] += myacc[i];
                free(myacc);
            }
            tot.crossings += T.crossings;
            tot.rays += T.rays;
            tot.near_tie_rays += T.near_tie_rays;
            tot.destroy += T.destroy;
            if (T.level_reached > tot.level_reached) tot.level_reached = T.level_reached;
            for (int l = 0; l < OR_NLEVELS; ++l) tot.per_level[l] += T.per_level[l];
            tot.absorbed += T.absorbed;
            tot.escaped += T.escaped;
            tot.dropped += T.dropped;
            tot.absorbed_n += T.absorbed_n;
            tot.escaped_n += T.escaped_n;
            tot.dropped_n += T.dropped_n;
        }
    }
    if (nsrc == 0) tot.level_reached = 0;
    dstat[0] = Lin;
    dstat[1] = tot.absorbed;
    dstat[2] = tot.escaped;
    dstat[3] = tot.dropped;
    dstat[4] = Ln_in;
    dstat[5] = tot.absorbed_n;
    dstat[6] = tot.escaped_n;
    dstat[7] = tot.dropped_n;
    istat[0] = tot.crossings;
    istat[1] = tot.rays;
    istat[2] = tot.near_tie_rays;
    istat[3] = tot.destroy;
    istat[4] = (long long)nsrc * (12LL << (2 * lmax_glob));
    istat[5] = tot.level_reached;
    istat[6] = lmax_glob;
    istat[7] = 0;
    for (int l = 0; l < OR_NLEVELS; ++l) istat[8 + l] = tot.per_level[l];
    free(u);
    return 0;
}

/*
 * Segments of one ray (level, pixel) of a source at pos, from its r_start to its end with
 * the given entering L and tau: cells, physical lengths. Returns the number of segments
 * written (at most cap), or -1 on invalid input; *end_reason receives the end reason.
 */
int or_ray_segments(int nx, int ny, int nz, const double* lo, double dx, const float* nH0,
                    const float* nH, const double* pos, int level0, int level_cap, double m_ray,
                    double tau_max, double sigma_H, double sigma_d, const double* rot,
                    double d_max, int level, unsigned long long pix, double L, double tau,
                    long long* cells, double* ds, int cap, int* end_reason)
{
    or_problem P;
    if (or_setup(&P, nx, ny, nz, dx, nH0, nH, level0, level_cap, m_ray, tau_max, sigma_H,
                 sigma_d, rot, d_max))
        return -1;
    double u[3];
    if (or_source_cells(&P, 1, lo, pos, u)) return -1;
    int lm = or_level_max(&P, u);
    if (level < level0 || level > lm) return -1;
    or_ray ray = {level, (uint64_t)pix, L, tau, 0.0, 0.0};
    or_segvec sv = {NULL, 0, 0};
    or_tally T;
    memset(&T, 0, sizeof(T));
    int near = 0;
    *end_reason = or_walk(&P, u, &ray, lm, NULL, 0, 0, &sv, &T, &near);
    int m = (int)(sv.n < (size_t)cap ? sv.n : (size_t)cap);
    for (int i = 0; i < m; ++i) { cells[i] = sv.v[i].cell; ds[i] = sv.v[i].ds; }
    int total = (int)sv.n;
    free(sv.v);
    return total;
}

/* ------------------------------------------------------------------------------------- */
/* Reverse sweep for loss = sum_c (w_c Gamma_c + v_c . f_rad,c) (new; not in the paper)    */
/* ------------------------------------------------------------------------------------- */

/*
 * For a ray and its descendants returns S, the sum of their segments' loss terms
 *   w_c K G + q dL,   G = L_in ds phi(dtau),  dL = L_in (1 - e^-dtau),  q = KF (v_c . n),
 * with K = sigma_H / dV (Gamma per unit G) and KF = 1 / dV (force per unit momentum), and adds
 * to grad[c] the derivative of the loss with respect to log n_H0[c]:
 *   own term    (w_c K L_in ds phi'(dtau) + q L_in e^-dtau) dtauH
 *   later terms -S_after dtauH,
 * where S_after is the loss over every later segment of the ray and over all of its
 * descendants (their entering luminosity carries the factor e^-dtau of this segment).
 * v may be NULL (no force term). tau_max and the split points are held fixed.
 */
static double or_adjoint_tree(const or_problem* P, const double u[3], int lmax, or_ray ray,
                              const double* w, const double* v, int64_t ncell, double K,
                              double KF, double* grad)
{
    or_segvec sv = {NULL, 0, 0};
    or_tally T;
    memset(&T, 0, sizeof(T));
    int near = 0;
    or_ray end = ray;
    int reason = or_walk(P, u, &end, lmax, NULL, 0, 0, &sv, &T, &near);
    double n[3];
    or_direction(P, ray.level, ray.pix, n);
    double own = 0.0;
    for (size_t j = 0; j < sv.n; ++j) {
        const or_seg* g = &sv.v[j];
        own += w[g->cell] * K * g->Lin * g->ds * or_phi(g->dtau);
        if (v) {
            const double q = KF * (v[g->cell] * n[0] + v[ncell + g->cell] * n[1] +
                                   v[2 * ncell + g->cell] * n[2]);
            own += q * -g->Lin * expm1(-g->dtau);
        }
    }
    double sub = 0.0;
    if (reason == OR_END_SPLIT) {
        for (int k = 0; k < 4; ++k) {
            or_ray ch = {ray.level + 1, 4 * ray.pix + (uint64_t)k, 0.25 * end.L, end.tau, 0.0, 0.0};
            sub += or_adjoint_tree(P, u, lmax, ch, w, v, ncell, K, KF, grad);
        }
    }
    double total = own + sub;
    double after = total;
    for (size_t j = 0; j < sv.n; ++j) {
        const or_seg* g = &sv.v[j];
        double gj = w[g->cell] * K * g->Lin * g->ds * or_phi(g->dtau);
        double dj = w[g->cell] * K * g->Lin * g->ds * or_dphi(g->dtau);
        if (v) {
            const double q = KF * (v[g->cell] * n[0] + v[ncell + g->cell] * n[1] +
                                   v[2 * ncell + g->cell] * n[2]);
            gj += q * -g->Lin * expm1(-g->dtau);
            dj += q * g->Lin * exp(-g->dtau);
        }
        after -= gj;
        grad[g->cell] += g->dtauH * (dj - after);
    }
    free(sv.v);
    return total;
}

/*
 * Gradient of loss = sum_c (w_c Gamma_c + v_c . f_rad,c) with respect to log n_H0 (per cell,
 * into grad) and to each source luminosity (dL[s] = loss_s / L_s, the loss being linear in
 * L_s). v: 3*ncell values (x block, y block, z block) or NULL for the Gamma term alone.
 * Returns 0, or -1 on invalid input (including a source with L_s <= 0).
 */
int or_trace_adjoint(int nx, int ny, int nz, const double* lo, double dx, const float* nH0,
                     const float* nH, int nsrc, const double* pos, const double* L, int level0,
                     int level_cap, double m_ray, double tau_max, double sigma_H, double sigma_d,
                     const double* rot, double d_max, const double* w, const double* v,
                     double* grad, double* dL, double* loss, int nthreads)
{
    or_problem P;
    if (or_setup(&P, nx, ny, nz, dx, nH0, nH, level0, level_cap, m_ray, tau_max, sigma_H,
                 sigma_d, rot, d_max))
        return -1;
    double* u = (double*)malloc(sizeof(double) * 3 * (size_t)(nsrc > 0 ? nsrc : 1));
    if (or_source_cells(&P, nsrc, lo, pos, u)) { free(u); return -1; }
    for (int s = 0; s < nsrc; ++s)
        if (!(L[s] > 0)) { free(u); return -1; }
    const int64_t ncell = (int64_t)nx * ny * nz;
    memset(grad, 0, sizeof(double) * (size_t)ncell);
    const double K = sigma_H / (dx * dx * dx);
    const double KF = 1.0 / (dx * dx * dx);
    const long long nbase = 12LL << (2 * level0);
    double total = 0.0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int s = 0; s < nsrc; ++s) {
        int lm = or_level_max(&P, u + 3 * s);
        double ls = 0.0;
#pragma omp parallel reduction(+ : ls)
        {
            double* g = grad;
            int nt = 1;
#ifdef _OPENMP
            nt = omp_get_num_threads();
#endif
            if (nt > 1) g = (double*)calloc((size_t)ncell, sizeof(double));
#pragma omp for schedule(dynamic, 8)
            for (long long p = 0; p < nbase; ++p) {
                or_ray root = {level0, (uint64_t)p, L[s] / (double)nbase, 0.0, 0.0, 0.0};
                ls += or_adjoint_tree(&P, u + 3 * s, lm, root, w, v, ncell, K, KF, g);
            }
#pragma omp critical
            if (g != grad) {
                for (int64_t i = 0; i < ncell; ++i) grad[i] += g[i];
                free(g);
            }
        }
        dL[s] = ls / L[s];
        total += ls;
    }
    *loss = total;
    free(u);
    return 0;
}
