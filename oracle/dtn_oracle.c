/*
 * dtn_oracle.c -- plain, slow FP64 CPU oracle of the local BIE / walk-on-spheres
 * Dirichlet-to-Neumann method (Yan, Cai, Zeng, arXiv 1210.1491).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * Every function restates one step of the method in the order the paper gives
 * it, in double precision, with no blocking, fusion or reordering:
 *   - Philox4x32-10 counter RNG (Salmon et al., SC'11; not in the paper)
 *   - Gauss-Legendre rules (Sec. 5.1.2, Eq. bw83/bw85 use them on the hemisphere)
 *   - distance to the boundary and nearest boundary point (Sec. 2, WOS paragraph)
 *   - walk on spheres with an epsilon-shell, estimator Eq. bw87
 *   - whole-sphere Dirichlet Green's function with one Kelvin image (Sec. 4,
 *     image charge/location as in the text after Eq. bw26)
 *   - local BIE of the first kind, Eq. bw49-bw51, collocation (Sec. 5.2)
 *   - dense LU with partial pivoting
 *   - integral representation Eq. bw03 with the free-space G of Eq. bw05
 *
 * Parity status of every function is listed in the test suite; all functions
 * here are pinned (none is "parity unpinned").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

/* ===================================================================== RNG */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11).  One round: two 32x32->64 products of counter words 0
 * and 2 with the round multipliers; the new words are
 *   (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)),
 * and the key is bumped by the Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 21-bit uniform: the odd integer 2f + 1 times 2^-22, in (0,1), for a 21-bit
 * field f of a Philox block. */
double or_u01_21(uint32_t f) { return (double)(2u * (f & 0x1fffffu) + 1u) * 0x1p-22; }

/* The six 21-bit fields of one Philox block w[0..3]: the top 21 bits of each
 * word, then the low 11 bits of w[0] with the low 10 bits of w[1] above them,
 * and the same of w[2], w[3]. */
void or_fields21(const uint32_t w[4], uint32_t f[6])
{
    for (int i = 0; i < 4; ++i) f[i] = w[i] >> 11;
    f[4] = (w[0] & 0x7ffu) | ((w[1] & 0x3ffu) << 11);
    f[5] = (w[2] & 0x7ffu) | ((w[3] & 0x3ffu) << 11);
}

/* 53-bit uniform from two words: the odd integer (hi<<21 | lo>>11) | 1 times 2^-53. */
double or_u01_53(uint32_t hi, uint32_t lo)
{
    uint64_t v = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
    return (double)(v | 1ull) * 0x1p-53;
}

/* ========================================================= Gauss-Legendre */
/* n-point Gauss-Legendre rule on [-1,1], nodes ascending.  Newton's method on
 * P_n evaluated by the three-term recurrence (k+1)P_{k+1} = (2k+1)xP_k - kP_{k-1};
 * weight 2 / ((1-x^2) P_n'(x)^2). */
void or_gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            if (n == 0) p1 = 1.0;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1; p1 = p2;
            }
            /* p1 = P_n(z), p0 = P_{n-1}(z) */
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) {
                /* one more evaluation of the derivative at the final node */
                p0 = 1.0; p1 = z;
                for (int k = 1; k < n; ++k) {
                    double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                    p0 = p1; p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                break;
            }
        }
        /* node i counted from +1 downward; store ascending */
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* ================================================================ geometry */
/* Domain kinds: 0 ball interior, 1 box interior, 2 box minus boxes, and two
 * unbounded regions where a walk that leaves the truncation sphere of radius
 * `truncation` about `center` has gone to infinity (Sec. 4.1.3): 3 the half
 * space z > center[2]; 4 space outside the thin disk of radius `radius` about
 * `center` in the plane z = center[2] (Test 4); 5 space outside the sphere of
 * radius `radius` about `center` (Sec. 5.2, the R = 3 sphere). */
typedef struct {
    int kind;
    double center[3], radius;
    double lo[3], hi[3];
    int n_boxes;
    const double *boxes; /* n_boxes x 6: lo xyz, hi xyz */
    double truncation;
} or_geom;

/* Distance from x to the boundary of the region and the nearest boundary point
 * (the radius of the largest empty sphere of the WOS step, Sec. 2).
 * Ties take the lowest face / box index; the outer box comes before the wires. */
double or_distance(const or_geom *g, const double x[3], double nearest[3])
{
    if (g->kind == 3) {
        nearest[0] = x[0]; nearest[1] = x[1]; nearest[2] = g->center[2];
        return x[2] - g->center[2];
    }
    if (g->kind == 5) {
        double v[3] = {x[0] - g->center[0], x[1] - g->center[1], x[2] - g->center[2]};
        double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (r > 0.0) {
            for (int i = 0; i < 3; ++i) nearest[i] = g->center[i] + g->radius * v[i] / r;
        } else {
            nearest[0] = g->center[0]; nearest[1] = g->center[1];
            nearest[2] = g->center[2] + g->radius;
        }
        return r - g->radius;
    }
    if (g->kind == 4) {
        double dx = x[0] - g->center[0], dy = x[1] - g->center[1], dz = x[2] - g->center[2];
        double r = sqrt(dx * dx + dy * dy);
        nearest[2] = g->center[2];
        if (r <= g->radius) {
            nearest[0] = x[0]; nearest[1] = x[1];
            return fabs(dz);
        }
        nearest[0] = g->center[0] + g->radius * dx / r;
        nearest[1] = g->center[1] + g->radius * dy / r;
        return sqrt((r - g->radius) * (r - g->radius) + dz * dz);
    }
    if (g->kind == 0) {
        double v[3] = {x[0] - g->center[0], x[1] - g->center[1], x[2] - g->center[2]};
        double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (r > 0.0) {
            for (int i = 0; i < 3; ++i) nearest[i] = g->center[i] + g->radius * v[i] / r;
        } else {
            nearest[0] = g->center[0]; nearest[1] = g->center[1];
            nearest[2] = g->center[2] + g->radius;
        }
        return g->radius - r;
    }
    /* outer box, interior side: face f = 2*axis + side */
    double best = INFINITY;
    int bf = 0;
    for (int f = 0; f < 6; ++f) {
        int ax = f / 2;
        double d = (f % 2 == 0) ? x[ax] - g->lo[ax] : g->hi[ax] - x[ax];
        if (d < best) { best = d; bf = f; }
    }
    nearest[0] = x[0]; nearest[1] = x[1]; nearest[2] = x[2];
    nearest[bf / 2] = (bf % 2 == 0) ? g->lo[bf / 2] : g->hi[bf / 2];
    if (g->kind == 1) return best;
    /* obstacle boxes, exterior side: |max(lo - x, 0, x - hi)| */
    for (int b = 0; b < g->n_boxes; ++b) {
        const double *lo = g->boxes + 6 * b, *hi = lo + 3;
        double e[3], s = 0.0;
        for (int i = 0; i < 3; ++i) {
            double t = lo[i] - x[i];
            double u = x[i] - hi[i];
            e[i] = t > 0.0 ? t : (u > 0.0 ? u : 0.0);
            s += e[i] * e[i];
        }
        double d = sqrt(s);
        if (d < best) {
            best = d;
            for (int i = 0; i < 3; ++i)
                nearest[i] = x[i] < lo[i] ? lo[i] : (x[i] > hi[i] ? hi[i] : x[i]);
        }
    }
    return best;
}

/* ============================================================ Dirichlet data */
typedef struct {
    int kind;              /* 0 point source, 1 harmonic polynomial (real SH), 2 constant */
    double x0[3], strength;
    int lmax;
    const double *clm;     /* (lmax+1)^2, index l*l + l + m */
    double center[3], scale;
    double constant;
} or_data;

/* Real orthonormal spherical harmonics Y_lm(direction), l <= lmax, index
 * l*l + l + m, no Condon-Shortley phase:
 *   m = 0 : N_l0 P_l(cos t)
 *   m > 0 : sqrt2 N_lm P_l^m(cos t) cos(m p)
 *   m < 0 : sqrt2 N_l|m| P_l^|m|(cos t) sin(|m| p)
 * with N_lm = sqrt((2l+1)/(4pi) (l-m)!/(l+m)!).  P_l^m by the recurrences
 * P_m^m = (2m-1)!! sin^m t,  P_{m+1}^m = (2m+1) cos t P_m^m,
 * (l-m) P_l^m = (2l-1) cos t P_{l-1}^m - (l+m-1) P_{l-2}^m. */
void or_real_sh(int lmax, const double dir[3], double *Y)
{
    double r = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    double ct = r > 0 ? dir[2] / r : 1.0;
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = atan2(dir[1], dir[0]);
    for (int m = 0; m <= lmax; ++m) {
        /* P_m^m */
        double pmm = 1.0;
        for (int k = 1; k <= m; ++k) pmm *= (2.0 * k - 1.0) * st;
        double plm2 = 0.0, plm1 = 0.0;
        for (int l = m; l <= lmax; ++l) {
            double p;
            if (l == m) p = pmm;
            else if (l == m + 1) p = (2.0 * m + 1.0) * ct * pmm;
            else p = ((2.0 * l - 1.0) * ct * plm1 - (l + m - 1.0) * plm2) / (double)(l - m);
            plm2 = plm1; plm1 = p;
            /* N_lm via the factorial ratio */
            double ratio = 1.0;
            for (int k = l - m + 1; k <= l + m; ++k) ratio /= (double)k;
            double N = sqrt((2.0 * l + 1.0) / (4.0 * OR_PI) * ratio);
            if (m == 0) {
                Y[l * l + l] = N * p;
            } else {
                Y[l * l + l + m] = sqrt(2.0) * N * p * cos(m * ph);
                Y[l * l + l - m] = sqrt(2.0) * N * p * sin(m * ph);
            }
        }
    }
}

/* Dirichlet data g(x) (the boundary values of u in Eq. bw01). */
double or_dirichlet(const or_data *d, const double x[3])
{
    if (d->kind == 0) {
        double v[3] = {x[0] - d->x0[0], x[1] - d->x0[1], x[2] - d->x0[2]};
        return d->strength / (4.0 * OR_PI * sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
    }
    if (d->kind == 1) {
        double v[3] = {(x[0] - d->center[0]) / d->scale, (x[1] - d->center[1]) / d->scale,
                       (x[2] - d->center[2]) / d->scale};
        double rho = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        int nl = (d->lmax + 1) * (d->lmax + 1);
        double Y[(32 + 1) * (32 + 1)];
        if (d->lmax > 32) return NAN;
        or_real_sh(d->lmax, v, Y);
        (void)nl;
        double s = 0.0, rl = 1.0;
        for (int l = 0; l <= d->lmax; ++l) {
            for (int m = -l; m <= l; ++m) s += d->clm[l * l + l + m] * rl * Y[l * l + l + m];
            rl *= rho;
        }
        return s;
    }
    return d->constant;
}

/* Exact Neumann data n . grad u for the harmonic extension of the data.
 * Point source: grad of strength/(4 pi |x-x0|).  Harmonic polynomial of degree
 * lmax: u restricted to the line x + t n is a polynomial of degree <= lmax, so
 * the central difference of order 2m >= lmax (weights (-1)^(k+1) (m!)^2 /
 * (k (m-k)! (m+k)!)) is exact for it. */
double or_neumann_exact(const or_data *d, const double x[3], const double n[3])
{
    if (d->kind == 0) {
        double v[3] = {x[0] - d->x0[0], x[1] - d->x0[1], x[2] - d->x0[2]};
        double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        return -d->strength * (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / (4.0 * OR_PI * r * r * r);
    }
    if (d->kind == 1) {
        int m = (d->lmax + 1) / 2 + 1;
        double h = 0.125 * d->scale;
        double mf = 1.0;
        for (int k = 1; k <= m; ++k) mf *= k;
        double s = 0.0;
        for (int k = 1; k <= m; ++k) {
            double fmk = 1.0, fpk = 1.0;
            for (int j = 1; j <= m - k; ++j) fmk *= j;
            for (int j = 1; j <= m + k; ++j) fpk *= j;
            double wk = ((k % 2) ? 1.0 : -1.0) * mf * mf / (k * fmk * fpk);
            double xp[3], xm[3];
            for (int i = 0; i < 3; ++i) { xp[i] = x[i] + k * h * n[i]; xm[i] = x[i] - k * h * n[i]; }
            s += wk * (or_dirichlet(d, xp) - or_dirichlet(d, xm));
        }
        return s / h;
    }
    return 0.0;
}

/* ==================================================================== WOS */
typedef struct {
    double eps;          /* absorption shell width */
    uint64_t seed;       /* Philox key = (seed lo32, seed hi32) */
    uint64_t max_steps;  /* distance evaluations per walk before a walk is cut */
    int stream;          /* 0: one Philox call per jump, 53-bit uniforms from words (0,1),(2,3)
                            1: one Philox call per three jumps, 21-bit uniforms; jump j uses
                               counter (walk, j/3, point, patch) and fields (2m, 2m+1), m = j%3,
                               of or_fields21 */
    int score;           /* 0: g at the nearest boundary point; 1: the data function at the
                            absorption point itself (martingale diagnostic) */
} or_wos_opts;

/* Uniform direction on the unit sphere from two uniforms (Sec. 2: the next
 * point of a walk is uniform on the sphere of radius d): z = 1 - 2 u1 is
 * uniform in (-1, 1) and the azimuth is uniform over a full turn, by
 * Archimedes' hat-box theorem.  Stream 0 takes the azimuth 2 pi u2 in (0, 2 pi);
 * stream 1 takes 2 pi (u2 - 1/2) in (-pi, pi), the same uniform law shifted by
 * half a turn (reading R3: the form the FP32 walks use, where u2 - 1/2 is exact
 * and needs no range reduction). */
static void direction_parts(double u1, double u2, int stream, double *z, double *s, double *ph)
{
    *z = 1.0 - 2.0 * u1;
    *s = sqrt(fmax(0.0, 1.0 - *z * *z));
    *ph = (stream == 0) ? 2.0 * OR_PI * u2 : 2.0 * OR_PI * (u2 - 0.5);
}

void or_direction(double u1, double u2, int stream, double om[3])
{
    double z, s, ph;
    direction_parts(u1, u2, stream, &z, &s, &ph);
    om[0] = s * cos(ph);
    om[1] = s * sin(ph);
    om[2] = z;
}

/* One walk on spheres (Sec. 2): from y, repeat { d = dist(x); stop if d <= eps;
 * jump to a uniform point of the sphere of radius d about x }.  Returns 1 and the
 * score when absorbed, 0 when the walk reached max_steps distance evaluations.
 * Unbounded regions (kinds 3, 4, 5): before each distance evaluation, a walk
 * outside the truncation sphere has gone to infinity and scores 0 (the
 * solution vanishes there). */
int or_walk(const or_geom *g, const or_data *dat, const double y[3], uint32_t walk,
            uint32_t point, uint32_t patch, const or_wos_opts *o, double *score, uint64_t *steps)
{
    double x[3] = {y[0], y[1], y[2]};
    uint32_t key[2] = {(uint32_t)(o->seed & 0xffffffffu), (uint32_t)(o->seed >> 32)};
    *steps = 0;
    for (uint64_t j = 0; j < o->max_steps; ++j) {
        double nb[3];
        if (g->kind >= 3) {
            double v[3] = {x[0] - g->center[0], x[1] - g->center[1], x[2] - g->center[2]};
            if (v[0] * v[0] + v[1] * v[1] + v[2] * v[2] > g->truncation * g->truncation) {
                *score = 0.0;
                return 1;
            }
        }
        double d = or_distance(g, x, nb);
        *steps += 1;
        if (d <= o->eps) {
            *score = (o->score == 0) ? or_dirichlet(dat, nb) : or_dirichlet(dat, x);
            return 1;
        }
        double u1, u2;
        uint32_t w[4];
        if (o->stream == 0) {
            uint32_t ctr[4] = {walk, (uint32_t)j, point, patch};
            or_philox4x32_10(ctr, key, w);
            u1 = or_u01_53(w[0], w[1]);
            u2 = or_u01_53(w[2], w[3]);
        } else {
            uint32_t ctr[4] = {walk, (uint32_t)(j / 3), point, patch};
            or_philox4x32_10(ctr, key, w);
            uint32_t f[6];
            or_fields21(w, f);
            int m = (int)(j % 3);
            u1 = or_u01_21(f[2 * m]);
            u2 = or_u01_21(f[2 * m + 1]);
        }
        double z, s, ph;
        direction_parts(u1, u2, o->stream, &z, &s, &ph);
        x[0] += d * s * cos(ph);
        x[1] += d * s * sin(ph);
        x[2] += d * z;
    }
    return 0;
}

/* Estimator Eq. bw87 at one hemisphere node: sums over walks [w0, w1). */
void or_wos_point(const or_geom *g, const or_data *dat, const double y[3], uint32_t point,
                  uint32_t patch, int64_t w0, int64_t w1, const or_wos_opts *o, double *sum,
                  double *sum2, uint64_t *steps, uint64_t *capped)
{
    double s1 = 0.0, s2 = 0.0;
    uint64_t st = 0, cap = 0;
    for (int64_t w = w0; w < w1; ++w) {
        double sc;
        uint64_t ns;
        if (or_walk(g, dat, y, (uint32_t)w, point, patch, o, &sc, &ns)) {
            s1 += sc;
            s2 += sc * sc;
        } else {
            cap += 1;
        }
        st += ns;
    }
    *sum = s1; *sum2 = s2; *steps = st; *capped = cap;
}

/* Many nodes at once (OpenMP over nodes; each node is the serial loop above). */
void or_wos_points(const or_geom *g, const or_data *dat, int64_t n, const double *y,
                   const uint32_t *point, const uint32_t *patch, const int64_t *walks,
                   const or_wos_opts *o, double *sum, double *sum2, uint64_t *steps,
                   uint64_t *capped)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i)
        or_wos_point(g, dat, y + 3 * i, point[i], patch[i], 0, walks[i], o, sum + i, sum2 + i,
                     steps + i, capped + i);
}

/* ================================================================ patches */
/* Patch kinds: 0 flat disk (S lies in one plane face), 1 spherical cap (S lies
 * on the boundary sphere of a ball domain), 2 wrapped box patch (the ball
 * about a point of an obstacle box's face meets several faces of that box: S
 * is made of face pieces, reading R15).  Local frame (t1, t2, n): n is the
 * outward normal of the region at c; t1 = normalised projection of the
 * coordinate axis least aligned with n (lowest index on ties); t2 = n x t1. */
#define OR_MAX_PIECES 6
#define OR_MAX_SUB 16

/* One piece of a wrapped patch: a face rectangle of the box cut by the ball,
 * i.e. rectangle intersect disk (the ball's slice of the face plane), a convex
 * region described in polar coordinates (rho, phi) about P, its point nearest
 * the disk centre (moved onto a rectangle side closer than rf/4, see
 * make_piece): rho <= rho_max(phi) for phi in [sub[0], sub[nsub]].  The
 * angle range is cut at the angles where rho_max changes from one rectangle
 * side or the circle to another, so rho_max is smooth between cuts. */
typedef struct {
    int ax, side;             /* the face: coordinate axis, 0 the lo face, 1 the hi face */
    int ua, va;               /* in-plane axes, ua < va */
    double fv;                /* the plane's coordinate along ax */
    double rlo[2], rhi[2];    /* the face rectangle in (ua, va) */
    double cf[2], rf;         /* the ball's slice of the plane: centre, radius */
    double P[2];              /* polar origin */
    int onlo[2], onhi[2];     /* P lies on the rectangle side u = rlo / rhi (then that side
                                 bounds no ray of the range) */
    int nsub;                 /* sub-ranges of the angle */
    double sub[OR_MAX_SUB + 1];
    double area;
} or_piece;

typedef struct {
    int kind;
    double c[3], n[3], t1[3], t2[3];
    double a;
    double R, sc[3];   /* cap: signed sphere radius (the sphere's centre is at c - R n:
                          R > 0 for a ball region, R < 0 outside a sphere) and centre */
    double theta_max;  /* hemisphere polar range measured from -n (kinds 0, 1) */
    double umax;       /* panel radial parameter range: a (disk) or psi_max (cap) */
    double blo[3], bhi[3];   /* wrapped patch: the obstacle box */
    int npiece;
    or_piece piece[OR_MAX_PIECES];
} or_patch;

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static void frame_from_normal(or_patch *p)
{
    int ax = 0;
    for (int i = 1; i < 3; ++i)
        if (fabs(p->n[i]) < fabs(p->n[ax])) ax = i;
    double e[3] = {0, 0, 0};
    e[ax] = 1.0;
    double en = p->n[ax];
    double t[3] = {e[0] - en * p->n[0], e[1] - en * p->n[1], e[2] - en * p->n[2]};
    double tn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    for (int i = 0; i < 3; ++i) p->t1[i] = t[i] / tn;
    cross3(p->n, p->t1, p->t2);
}

/* ----------------------------------------------------- wrapped box patches */
/* rho_max(phi) of a piece: the distance from P along (cos phi, sin phi) to the
 * circle, or to a rectangle side if one is nearer (sides through P excepted). */
static double piece_rho(const or_piece *q, double ph)
{
    const double e[2] = {cos(ph), sin(ph)};
    const double w0 = q->P[0] - q->cf[0], w1 = q->P[1] - q->cf[1];
    const double we = w0 * e[0] + w1 * e[1], ww = w0 * w0 + w1 * w1;
    double r = -we + sqrt(fmax(0.0, we * we - ww + q->rf * q->rf));
    for (int k = 0; k < 2; ++k) {
        if (e[k] > 0.0 && !q->onhi[k]) r = fmin(r, (q->rhi[k] - q->P[k]) / e[k]);
        if (e[k] < 0.0 && !q->onlo[k]) r = fmin(r, (q->rlo[k] - q->P[k]) / e[k]);
    }
    return r;
}

static int cmp_double(const void *x, const void *y)
{
    const double a = *(const double *)x, b = *(const double *)y;
    return (a > b) - (a < b);
}

/* The piece of box face f (axis f/2, lo face for f even) inside the ball
 * B(c, a); 0 if the ball does not meet the closed face rectangle. */
static int make_piece(const double lo[3], const double hi[3], int f, const double c[3], double a,
                      or_piece *q)
{
    memset(q, 0, sizeof(*q));
    q->ax = f / 2;
    q->side = f % 2;
    q->fv = q->side ? hi[q->ax] : lo[q->ax];
    const double d = c[q->ax] - q->fv;
    if (!(fabs(d) < a)) return 0;
    q->ua = (q->ax == 0) ? 1 : 0;
    q->va = (q->ax == 2) ? 1 : 2;
    const int ax2[2] = {q->ua, q->va};
    for (int k = 0; k < 2; ++k) {
        q->rlo[k] = lo[ax2[k]];
        q->rhi[k] = hi[ax2[k]];
        q->cf[k] = c[ax2[k]];
        q->P[k] = fmin(fmax(q->cf[k], q->rlo[k]), q->rhi[k]);
    }
    q->rf = sqrt(a * a - d * d);
    {
        /* a polar origin closer than rf/4 to a rectangle side moves onto that
         * side (onto the corner when near two), as long as it stays well inside
         * the disk: the rays from P would otherwise cross a thin strip between
         * P and the side, whose rings are sliver panels (aspect ratios in the
         * thousands, collocation systems with condition numbers 1e3 and more) */
        const double snap = 0.25 * q->rf;
        for (int k = 0; k < 2; ++k) {
            const double dl = q->P[k] - q->rlo[k], dh = q->rhi[k] - q->P[k];
            const double t = dl <= dh ? q->rlo[k] : q->rhi[k];
            if ((dl <= dh ? dl : dh) < snap) {
                double Pt[2] = {q->P[0], q->P[1]};
                Pt[k] = t;
                if (hypot(Pt[0] - q->cf[0], Pt[1] - q->cf[1]) < 0.9 * q->rf) q->P[k] = t;
            }
        }
    }
    for (int k = 0; k < 2; ++k) {
        q->onlo[k] = (q->P[k] == q->rlo[k]);
        q->onhi[k] = (q->P[k] == q->rhi[k]);
    }
    const double dP = hypot(q->P[0] - q->cf[0], q->P[1] - q->cf[1]);
    if (!(dP < q->rf)) return 0;
    /* the angles of the rays from P into the rectangle: every side through P
     * halves the range (quarter at a corner) */
    double ph0 = 0.0, ph1 = 2.0 * OR_PI;
    if (q->onlo[0] && q->onlo[1]) { ph0 = 0.0; ph1 = 0.5 * OR_PI; }
    else if (q->onhi[0] && q->onlo[1]) { ph0 = 0.5 * OR_PI; ph1 = OR_PI; }
    else if (q->onhi[0] && q->onhi[1]) { ph0 = OR_PI; ph1 = 1.5 * OR_PI; }
    else if (q->onlo[0] && q->onhi[1]) { ph0 = 1.5 * OR_PI; ph1 = 2.0 * OR_PI; }
    else if (q->onlo[0]) { ph0 = -0.5 * OR_PI; ph1 = 0.5 * OR_PI; }
    else if (q->onhi[0]) { ph0 = 0.5 * OR_PI; ph1 = 1.5 * OR_PI; }
    else if (q->onlo[1]) { ph0 = 0.0; ph1 = OR_PI; }
    else if (q->onhi[1]) { ph0 = OR_PI; ph1 = 2.0 * OR_PI; }
    /* cuts: the directions of the rectangle corners inside the disk and of the
     * points where the circle crosses a rectangle side */
    double cut[12];
    int nc = 0;
    double pts[12][2];
    int np = 0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            const double Q[2] = {i ? q->rhi[0] : q->rlo[0], j ? q->rhi[1] : q->rlo[1]};
            if (hypot(Q[0] - q->cf[0], Q[1] - q->cf[1]) < q->rf) { pts[np][0] = Q[0]; pts[np][1] = Q[1]; ++np; }
        }
    for (int k = 0; k < 2; ++k) {        /* sides u_k = const */
        const int o = 1 - k;
        for (int sd = 0; sd < 2; ++sd) {
            const double uk = sd ? q->rhi[k] : q->rlo[k];
            const double h2 = q->rf * q->rf - (uk - q->cf[k]) * (uk - q->cf[k]);
            if (!(h2 > 0.0)) continue;
            for (int sg = -1; sg <= 1; sg += 2) {
                const double vo = q->cf[o] + sg * sqrt(h2);
                if (vo > q->rlo[o] && vo < q->rhi[o]) {
                    pts[np][k] = uk; pts[np][o] = vo; ++np;
                }
            }
        }
    }
    for (int i = 0; i < np; ++i) {
        const double dx = pts[i][0] - q->P[0], dy = pts[i][1] - q->P[1];
        if (hypot(dx, dy) < 1e-12 * q->rf) continue;
        double ang = atan2(dy, dx);
        while (ang < ph0) ang += 2.0 * OR_PI;
        while (ang >= ph0 + 2.0 * OR_PI) ang -= 2.0 * OR_PI;
        if (ang > ph0 + 1e-12 && ang < ph1 - 1e-12) cut[nc++] = ang;
    }
    qsort(cut, nc, sizeof(double), cmp_double);
    q->sub[0] = ph0;
    q->nsub = 0;
    for (int i = 0; i < nc; ++i)
        if (cut[i] - q->sub[q->nsub] > 1e-12) q->sub[++q->nsub] = cut[i];
    if (ph1 - q->sub[q->nsub] > 1e-12) q->sub[++q->nsub] = ph1;
    else q->sub[q->nsub] = ph1;
    /* area: int 1/2 rho_max^2 dphi, 32-point Gauss per sub-range */
    double gx[32], gw[32];
    or_gauss_legendre(32, gx, gw);
    q->area = 0.0;
    for (int j = 0; j < q->nsub; ++j) {
        const double h = 0.5 * (q->sub[j + 1] - q->sub[j]), m = 0.5 * (q->sub[j + 1] + q->sub[j]);
        for (int i = 0; i < 32; ++i) {
            const double r = piece_rho(q, m + h * gx[i]);
            q->area += gw[i] * h * 0.5 * r * r;
        }
    }
    return 1;
}

/* Point of the hemisphere Gamma at polar angle th (from -n) and azimuth ph. */
static void arc_point(const or_patch *p, double th, double ph, double y[3])
{
    const double L[3] = {p->a * sin(th) * cos(ph), p->a * sin(th) * sin(ph), -p->a * cos(th)};
    for (int i = 0; i < 3; ++i) y[i] = p->c[i] + L[0] * p->t1[i] + L[1] * p->t2[i] + L[2] * p->n[i];
}

static int in_box(const double lo[3], const double hi[3], const double y[3])
{
    return y[0] >= lo[0] && y[0] <= hi[0] && y[1] >= lo[1] && y[1] <= hi[1] && y[2] >= lo[2] && y[2] <= hi[2];
}

/* Wrapped patch (R4): theta_max(ph) is where the great-circle arc from the
 * pole -n at azimuth ph first leaves the region, i.e. enters the box.  The
 * arc lies outside the box for theta < pi/2 (the box is on the +n side of the
 * face plane); on [pi/2, pi] it is sampled at 4096 points and the first entry
 * bracketed and bisected to 1e-15.  *star = 0 if a later sample is outside the
 * box again (the arc re-enters the region: Gamma is not star-shaped about the
 * pole, and the patch is not supported). */
static double theta_max_box(const or_patch *p, double ph, int *star)
{
    const int M = 4096;
    double y[3];
    double th_in = -1.0, th_out = 0.5 * OR_PI;
    for (int m = 0; m <= M; ++m) {
        const double th = 0.5 * OR_PI * (1.0 + (double)m / M);
        arc_point(p, th, ph, y);
        const int in = in_box(p->blo, p->bhi, y);
        if (th_in < 0.0) {
            if (in) th_in = th;
            else th_out = th;
        } else if (!in) {
            *star = 0;
        }
    }
    if (th_in < 0.0) {   /* never enters the box: the arc runs out of the ball's reach */
        *star = 0;
        return OR_PI;
    }
    if (th_in == 0.5 * OR_PI) return th_in;
    double lo = th_out, hi = th_in;   /* lo outside, hi inside */
    while (hi - lo > 1e-15) {
        const double mid = 0.5 * (lo + hi);
        arc_point(p, mid, ph, y);
        if (in_box(p->blo, p->bhi, y)) hi = mid;
        else lo = mid;
        if (mid == lo && mid == hi) break;
    }
    return hi;
}

/* Returns 0 on success, -1 if the ball about c meets more than one plane face
 * or the geometry/centre combination is not supported. */
int or_patch_frame(const or_geom *g, const double c[3], double a, or_patch *p)
{
    memset(p, 0, sizeof(*p));
    for (int i = 0; i < 3; ++i) p->c[i] = c[i];
    p->a = a;
    if (g->kind == 0) {
        double v[3] = {c[0] - g->center[0], c[1] - g->center[1], c[2] - g->center[2]};
        double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (!(a < 2.0 * g->radius) || r == 0.0) return -1;
        for (int i = 0; i < 3; ++i) { p->n[i] = v[i] / r; p->sc[i] = g->center[i]; }
        p->kind = 1;
        p->R = g->radius;
        /* |y - centre| <= R on the hemisphere  <=>  cos(theta) >= a / (2R) */
        p->theta_max = acos(a / (2.0 * g->radius));
        /* geodesic angle of the cap: chord a  <=>  psi = 2 asin(a / 2R) */
        p->umax = 2.0 * asin(a / (2.0 * g->radius));
        frame_from_normal(p);
        return 0;
    }
    if (g->kind == 3 || g->kind == 4) {
        /* the plane z = center[2] (half space: the region lies above it; thin
         * disk: the top face, with the ball's slice of the plane inside the disk) */
        if (!(fabs(c[2] - g->center[2]) <= 1e-9 * fmax(1.0, fabs(g->center[2])))) return -1;
        if (g->kind == 4) {
            double dx = c[0] - g->center[0], dy = c[1] - g->center[1];
            if (!(sqrt(dx * dx + dy * dy) + a < g->radius)) return -1;
        }
        p->n[0] = 0.0; p->n[1] = 0.0; p->n[2] = -1.0;
        p->kind = 0;
        p->theta_max = OR_PI / 2.0;
        p->umax = a;
        frame_from_normal(p);
        return 0;
    }
    if (g->kind == 5) {
        /* outside a sphere: the outward normal of the region points into the
         * sphere, whose centre lies at c + R_sphere n, i.e. signed R = -R_sphere */
        double v[3] = {c[0] - g->center[0], c[1] - g->center[1], c[2] - g->center[2]};
        double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (!(a < 2.0 * g->radius) || !(fabs(r - g->radius) <= 1e-9 * g->radius)) return -1;
        for (int i = 0; i < 3; ++i) { p->n[i] = -v[i] / r; p->sc[i] = g->center[i]; }
        p->kind = 1;
        p->R = -g->radius;
        /* |y - centre| >= R on the hemisphere  <=>  cos(theta) >= -a / (2R) */
        p->theta_max = OR_PI - acos(a / (2.0 * g->radius));
        p->umax = 2.0 * asin(a / (2.0 * g->radius));
        frame_from_normal(p);
        return 0;
    }
    /* plane faces: find the face containing c */
    double best = INFINITY;
    int bw = -2, bf = -1;
    for (int f = 0; f < 6; ++f) {
        int ax = f / 2;
        double d = fabs((f % 2 == 0) ? c[ax] - g->lo[ax] : g->hi[ax] - c[ax]);
        if (d < best) { best = d; bw = -1; bf = f; }
    }
    if (g->kind == 2) {
        for (int b = 0; b < g->n_boxes; ++b) {
            const double *lo = g->boxes + 6 * b, *hi = lo + 3;
            for (int f = 0; f < 6; ++f) {
                int ax = f / 2;
                double d = fabs((f % 2 == 0) ? c[ax] - lo[ax] : c[ax] - hi[ax]);
                /* c must lie within the face rectangle */
                int in = 1;
                for (int i = 0; i < 3; ++i)
                    if (i != ax && (c[i] < lo[i] || c[i] > hi[i])) in = 0;
                if (in && d < best) { best = d; bw = b; bf = f; }
            }
        }
    }
    int ax = bf / 2, side = bf % 2;
    p->n[0] = p->n[1] = p->n[2] = 0.0;
    if (bw == -1) p->n[ax] = side ? 1.0 : -1.0;   /* outer box: outward of the box */
    else p->n[ax] = side ? -1.0 : 1.0;            /* obstacle: region normal points into the box */
    p->kind = 0;
    p->theta_max = OR_PI / 2.0;
    p->umax = a;
    frame_from_normal(p);
    /* the ball must meet this face only */
    if (bw == -1) {
        for (int f = 0; f < 6; ++f) {
            if (f == bf) continue;
            int fx = f / 2;
            double d = (f % 2 == 0) ? c[fx] - g->lo[fx] : g->hi[fx] - c[fx];
            if (d <= a) return -1;
        }
    } else {
        const double *lo = g->boxes + 6 * bw, *hi = lo + 3;
        /* the ball must not reach the outer box (another conductor) */
        for (int f = 0; f < 6; ++f) {
            int fx = f / 2;
            double d = (f % 2 == 0) ? c[fx] - g->lo[fx] : g->hi[fx] - c[fx];
            if (d <= a) return -1;
        }
        int wrap = (hi[ax] - lo[ax] <= a);
        for (int i = 0; i < 3; ++i)
            if (i != ax && (c[i] - lo[i] <= a || hi[i] - c[i] <= a)) wrap = 1;
        if (wrap) {
            /* the ball meets further faces of this box: a wrapped patch made of
             * the face pieces inside the ball (R15), with Gamma star-shaped about
             * the pole */
            p->kind = 2;
            for (int i = 0; i < 3; ++i) { p->blo[i] = lo[i]; p->bhi[i] = hi[i]; }
            p->npiece = 0;
            for (int f = 0; f < 6; ++f) {
                /* the face containing c first, then the others in face order */
                int ff = (f == 0) ? bf : (f <= bf ? f - 1 : f);
                or_piece q;
                if (make_piece(lo, hi, ff, c, a, &q)) {
                    if (q.nsub > OR_MAX_SUB) return -1;
                    p->piece[p->npiece++] = q;
                }
            }
            p->theta_max = 0.0;
            p->umax = 0.0;
        }
    }
    if (g->kind == 2) {
        for (int b = 0; b < g->n_boxes; ++b) {
            if (b == bw) continue;
            const double *lo = g->boxes + 6 * b, *hi = lo + 3;
            double s = 0.0;
            for (int i = 0; i < 3; ++i) {
                double t = fmax(fmax(lo[i] - c[i], 0.0), c[i] - hi[i]);
                s += t * t;
            }
            if (sqrt(s) <= a) return -1;
        }
    }
    if (p->kind == 2) {
        /* Gamma must be star-shaped about the pole: probe 256 azimuths */
        int star = 1;
        for (int j = 0; j < 256 && star; ++j) theta_max_box(p, 2.0 * OR_PI * (j + 0.5) / 256, &star);
        if (!star) return -1;
    }
    return 0;
}

static void local_to_global(const or_patch *p, const double L[3], double y[3])
{
    for (int i = 0; i < 3; ++i) y[i] = p->c[i] + L[0] * p->t1[i] + L[1] * p->t2[i] + L[2] * p->n[i];
}

/* Hemisphere nodes (Eq. bw85 generalised to theta in [0, theta_max]; on a
 * wrapped patch theta_max depends on the azimuth, reading R4):
 * theta_i = (theta_max/2)(xi_i + 1), phi_j = pi (xi_j + 1), node index i*nphi + j,
 * local position a (sin th cos ph, sin th sin ph, -cos th), weight
 * w_i w_j (theta_max/2) pi a^2 sin th_i (the area element of Eq. bw83). */
void or_gamma_nodes(const or_patch *p, int nt, int nph, double *Yloc, double *yglob, double *W)
{
    double *xt = malloc(sizeof(double) * nt), *wt = malloc(sizeof(double) * nt);
    double *xp = malloc(sizeof(double) * nph), *wp = malloc(sizeof(double) * nph);
    or_gauss_legendre(nt, xt, wt);
    or_gauss_legendre(nph, xp, wp);
    for (int j = 0; j < nph; ++j) {
        double ph = OR_PI * (xp[j] + 1.0);
        /* polar range of this azimuth: fixed (kinds 0, 1) or theta_max(ph) (kind 2) */
        int star = 1;
        double tmax = (p->kind == 2) ? theta_max_box(p, ph, &star) : p->theta_max;
        for (int i = 0; i < nt; ++i) {
            double th = 0.5 * tmax * (xt[i] + 1.0);
            int k = i * nph + j;
            double L[3] = {p->a * sin(th) * cos(ph), p->a * sin(th) * sin(ph), -p->a * cos(th)};
            if (Yloc) { Yloc[3 * k] = L[0]; Yloc[3 * k + 1] = L[1]; Yloc[3 * k + 2] = L[2]; }
            if (yglob) local_to_global(p, L, yglob + 3 * k);
            W[k] = wt[i] * wp[j] * 0.5 * tmax * OR_PI * p->a * p->a * sin(th);
        }
    }
    free(xt); free(wt); free(xp); free(wp);
}

/* Point of the patch at parameters (u, v) (of piece `piece` on a wrapped patch),
 * local coordinates, its unit normal (local) and the area Jacobian.  Disk:
 * Y = u (cos v, sin v, 0), J = u.
 * Cap: Y = (R sin u cos v, R sin u sin v, -2R sin^2(u/2)), n = (sin u cos v,
 * sin u sin v, cos u), J = R^2 sin u. */
static void patch_point(const or_patch *p, int piece, double u, double v, double Y[3], double nl[3], double *J)
{
    if (p->kind == 2) {
        /* piece of a wrapped patch: u = rho / rho_max(v), v = phi; the point
         * P + u rho_max(v) (cos v, sin v) of the face plane; J = u rho_max(v)^2;
         * the normal points into the box (outward of the region) */
        const or_piece *q = &p->piece[piece];
        const double r = piece_rho(q, v);
        /* y - c formed from (P - c) and the offset, never from y itself: far
         * from the origin the global coordinates' spacing (1e-14 at 50) would
         * round a point next to the collocation point onto it */
        double d[3], ng[3] = {0.0, 0.0, 0.0};
        d[q->ax] = q->fv - p->c[q->ax];
        d[q->ua] = (q->P[0] - p->c[q->ua]) + u * r * cos(v);
        d[q->va] = (q->P[1] - p->c[q->va]) + u * r * sin(v);
        ng[q->ax] = q->side ? -1.0 : 1.0;
        Y[0] = d[0] * p->t1[0] + d[1] * p->t1[1] + d[2] * p->t1[2];
        Y[1] = d[0] * p->t2[0] + d[1] * p->t2[1] + d[2] * p->t2[2];
        Y[2] = d[0] * p->n[0] + d[1] * p->n[1] + d[2] * p->n[2];
        nl[0] = ng[0] * p->t1[0] + ng[1] * p->t1[1] + ng[2] * p->t1[2];
        nl[1] = ng[0] * p->t2[0] + ng[1] * p->t2[1] + ng[2] * p->t2[2];
        nl[2] = ng[0] * p->n[0] + ng[1] * p->n[1] + ng[2] * p->n[2];
        *J = u * r * r;
        return;
    }
    (void)piece;
    if (p->kind == 0) {
        Y[0] = u * cos(v); Y[1] = u * sin(v); Y[2] = 0.0;
        nl[0] = 0.0; nl[1] = 0.0; nl[2] = 1.0;
        *J = u;
    } else {
        double su = sin(u), cu = cos(u), sh = sin(0.5 * u);
        Y[0] = p->R * su * cos(v); Y[1] = p->R * su * sin(v); Y[2] = -2.0 * p->R * sh * sh;
        nl[0] = su * cos(v); nl[1] = su * sin(v); nl[2] = cu;
        *J = p->R * p->R * su;
    }
}

/* Panels: ring r in [0,nr), sector s in [0,ns), index r*ns + s; parameter box
 * u in [r umax/nr, (r+1) umax/nr], v in [s 2pi/ns, (s+1) 2pi/ns].
 * Collocation point = the panel's area centroid (disk), or the radial projection
 * of its area centroid onto the sphere (cap).  prm = (u0, u1, v0, v1, uc, vc,
 * piece), OR_PRM values per panel.
 * Wrapped patch (kind 2, R8): the ns sectors are shared among the sub-ranges of
 * all pieces (pieces in order, sub-ranges by angle) whose area is at least
 * area(S) / (nr^2 ns) (smaller ones get none and are left out of S): one
 * each, then one at a time to the sub-range with the largest area per sector
 * (a larger ratio wins
 * only by more than 1e-12 relative, else the lowest index), and a sub-range's
 * sectors split its angle evenly; rings split u =
 * rho / rho_max in [0, 1] evenly; the collocation point is the image of the
 * parameter box's midpoint.  Returns -1 if ns is below the number of
 * sub-ranges. */
#define OR_PRM 7
int or_panels(const or_patch *p, int nr, int ns, double *Xloc, double *xglob, double *nglob,
              double *area, double *prm)
{
    if (p->kind == 2) {
        int nsr = 0, pc[OR_MAX_PIECES * OR_MAX_SUB], sj[OR_MAX_PIECES * OR_MAX_SUB], cnt[OR_MAX_PIECES * OR_MAX_SUB];
        double sa[OR_MAX_PIECES * OR_MAX_SUB];
        double gx[32], gw[32];
        or_gauss_legendre(32, gx, gw);
        for (int k = 0; k < p->npiece; ++k)
            for (int j = 0; j < p->piece[k].nsub; ++j) {
                const or_piece *q = &p->piece[k];
                const double h = 0.5 * (q->sub[j + 1] - q->sub[j]), m = 0.5 * (q->sub[j + 1] + q->sub[j]);
                double A = 0.0;
                for (int i = 0; i < 32; ++i) {
                    const double r = piece_rho(q, m + h * gx[i]);
                    A += gw[i] * h * 0.5 * r * r;
                }
                pc[nsr] = k; sj[nsr] = j; sa[nsr] = A; cnt[nsr] = 1; ++nsr;
            }
        /* a sub-range whose area is below As / (nr^2 ns), less than a ring-0
         * panel of the patch split evenly, gets no sector: it is below the
         * layout's resolution (a ball that grazes a face, or a direction cut
         * next to a rectangle corner) and its rings would be slivers */
        double As = 0.0;
        for (int t = 0; t < nsr; ++t) As += sa[t];
        const double thr = As / ((double)nr * nr * ns);
        int used = 0, first = -1;
        for (int t = 0; t < nsr; ++t) {
            cnt[t] = sa[t] >= thr ? 1 : 0;
            used += cnt[t];
            if (cnt[t] && first < 0) first = t;
        }
        if (ns < used || first < 0) return -1;
        for (int extra = ns - used; extra > 0; --extra) {
            int best = first;
            for (int t = first + 1; t < nsr; ++t)
                if (cnt[t] && sa[t] / cnt[t] > sa[best] / cnt[best] * (1.0 + 1e-12)) best = t;
            cnt[best] += 1;
        }
        int sector = 0;
        for (int t = 0; t < nsr; ++t) {
            const or_piece *q = &p->piece[pc[t]];
            const double a0 = q->sub[sj[t]], a1 = q->sub[sj[t] + 1];
            for (int m = 0; m < cnt[t]; ++m, ++sector) {
                const double v0 = a0 + (a1 - a0) * m / cnt[t], v1 = a0 + (a1 - a0) * (m + 1) / cnt[t];
                const double vc = 0.5 * (v0 + v1);
                /* int_{v0}^{v1} rho_max^2 dv, for the panel areas */
                const double h = 0.5 * (v1 - v0);
                double R2 = 0.0;
                for (int i = 0; i < 32; ++i) {
                    const double r = piece_rho(q, vc + h * gx[i]);
                    R2 += gw[i] * h * r * r;
                }
                for (int r = 0; r < nr; ++r) {
                    const int k = r * ns + sector;
                    const double u0 = (double)r / nr, u1 = (double)(r + 1) / nr, uc = 0.5 * (u0 + u1);
                    double Y[3], nl[3], J;
                    patch_point(p, pc[t], uc, vc, Y, nl, &J);
                    if (Xloc) { Xloc[3 * k] = Y[0]; Xloc[3 * k + 1] = Y[1]; Xloc[3 * k + 2] = Y[2]; }
                    if (xglob) local_to_global(p, Y, xglob + 3 * k);
                    if (nglob)
                        for (int i = 0; i < 3; ++i)
                            nglob[3 * k + i] = nl[0] * p->t1[i] + nl[1] * p->t2[i] + nl[2] * p->n[i];
                    area[k] = 0.5 * (u1 * u1 - u0 * u0) * R2;
                    if (prm) {
                        double *w = prm + OR_PRM * k;
                        w[0] = u0; w[1] = u1; w[2] = v0; w[3] = v1; w[4] = uc; w[5] = vc; w[6] = pc[t];
                    }
                }
            }
        }
        return 0;
    }
    double du = p->umax / nr, dv = 2.0 * OR_PI / ns;
    double sinc = sin(0.5 * dv) / (0.5 * dv);
    for (int r = 0; r < nr; ++r) {
        for (int s = 0; s < ns; ++s) {
            int k = r * ns + s;
            double u0 = r * du, u1 = (r + 1) * du, v0 = s * dv, v1 = (s + 1) * dv;
            double vc = 0.5 * (v0 + v1), uc, A;
            if (p->kind == 0) {
                uc = (2.0 / 3.0) * (u1 * u1 * u1 - u0 * u0 * u0) / (u1 * u1 - u0 * u0) * sinc;
                A = 0.5 * (u1 * u1 - u0 * u0) * dv;
            } else {
                /* centroid direction: polar angle atan2(int sin^2 u du * sinc, int sin u cos u du) */
                double Is = 0.5 * ((u1 - sin(u1) * cos(u1)) - (u0 - sin(u0) * cos(u0)));
                double Ic = 0.5 * (sin(u1) * sin(u1) - sin(u0) * sin(u0));
                uc = atan2(Is * sinc, Ic);
                A = p->R * p->R * (cos(u0) - cos(u1)) * dv;
            }
            double Y[3], nl[3], J;
            patch_point(p, 0, uc, vc, Y, nl, &J);
            if (Xloc) { Xloc[3 * k] = Y[0]; Xloc[3 * k + 1] = Y[1]; Xloc[3 * k + 2] = Y[2]; }
            if (xglob) local_to_global(p, Y, xglob + 3 * k);
            if (nglob)
                for (int i = 0; i < 3; ++i)
                    nglob[3 * k + i] = nl[0] * p->t1[i] + nl[1] * p->t2[i] + nl[2] * p->n[i];
            area[k] = A;
            if (prm) {
                double *q = prm + OR_PRM * k;
                q[0] = u0; q[1] = u1; q[2] = v0; q[3] = v1; q[4] = uc; q[5] = vc; q[6] = 0.0;
            }
        }
    }
    return 0;
}

/* ======================================================= Green's functions */
/* Whole-sphere Dirichlet Green's function of B(c,a) in local coordinates
 * X = x - c, Y = y - c (Sec. 4: free-space term plus one Kelvin image of charge
 * -a/|Y| at c + a^2 Y/|Y|^2; written symmetrically in X and Y):
 *   G = (1/4pi) [ 1/|X-Y| - a / sqrt(|X|^2|Y|^2 - 2a^2 X.Y + a^4) ]. */
double or_green(double a, const double X[3], const double Y[3])
{
    double d[3] = {X[0] - Y[0], X[1] - Y[1], X[2] - Y[2]};
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double xx = X[0] * X[0] + X[1] * X[1] + X[2] * X[2];
    double yy = Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2];
    double xy = X[0] * Y[0] + X[1] * Y[1] + X[2] * Y[2];
    double Q = xx * yy - 2.0 * a * a * xy + a * a * a * a;
    return (1.0 / r - a / sqrt(Q)) / (4.0 * OR_PI);
}

/* grad_Y G = (1/4pi) [ (X-Y)/|X-Y|^3 + a (|X|^2 Y - a^2 X) / Q^{3/2} ]. */
void or_green_grad_y(double a, const double X[3], const double Y[3], double g[3])
{
    double d[3] = {X[0] - Y[0], X[1] - Y[1], X[2] - Y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double r3 = r2 * sqrt(r2);
    double xx = X[0] * X[0] + X[1] * X[1] + X[2] * X[2];
    double yy = Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2];
    double xy = X[0] * Y[0] + X[1] * Y[1] + X[2] * Y[2];
    double Q = xx * yy - 2.0 * a * a * xy + a * a * a * a;
    double Q32 = Q * sqrt(Q);
    for (int i = 0; i < 3; ++i)
        g[i] = (d[i] / r3 + a * (xx * Y[i] - a * a * X[i]) / Q32) / (4.0 * OR_PI);
}

/* Poisson kernel of B(c,a): -dG/dn_y on |Y| = a, = (a^2 - |X|^2) / (4 pi a |X-Y|^3)
 * (the hitting density of Eq. bw21 for the ball). */
double or_poisson(double a, const double X[3], const double Y[3])
{
    double d[3] = {X[0] - Y[0], X[1] - Y[1], X[2] - Y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double xx = X[0] * X[0] + X[1] * X[1] + X[2] * X[2];
    return (a * a - xx) / (4.0 * OR_PI * a * r2 * sqrt(r2));
}

/* Second normal derivative d2G/dn_x dn_y of the Green's function above (R1),
 * for unit normals nx at X and ny at Y (the kernel of Eq. bw53 and bw59):
 *   (1/4pi) [ nx.ny / r^3 - 3 (D.nx)(D.ny) / r^5
 *             + a ( (2 (X.nx)(Y.ny) - a^2 nx.ny) Q^{-3/2}
 *                   - 3 (|X|^2 Y.ny - a^2 X.ny)(|Y|^2 X.nx - a^2 Y.nx) Q^{-5/2} ) ],
 * D = X - Y, r = |D|, Q = |X|^2 |Y|^2 - 2 a^2 X.Y + a^4. */
double or_green_dnn(double a, const double X[3], const double nx[3], const double Y[3], const double ny[3])
{
    double D[3] = {X[0] - Y[0], X[1] - Y[1], X[2] - Y[2]};
    double r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2], r = sqrt(r2);
    double Dnx = D[0] * nx[0] + D[1] * nx[1] + D[2] * nx[2];
    double Dny = D[0] * ny[0] + D[1] * ny[1] + D[2] * ny[2];
    double nn = nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2];
    double XX = X[0] * X[0] + X[1] * X[1] + X[2] * X[2];
    double YY = Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2];
    double XY = X[0] * Y[0] + X[1] * Y[1] + X[2] * Y[2];
    double Xnx = X[0] * nx[0] + X[1] * nx[1] + X[2] * nx[2];
    double Yny = Y[0] * ny[0] + Y[1] * ny[1] + Y[2] * ny[2];
    double Xny = X[0] * ny[0] + X[1] * ny[1] + X[2] * ny[2];
    double Ynx = Y[0] * nx[0] + Y[1] * nx[1] + Y[2] * nx[2];
    double Q = XX * YY - 2.0 * a * a * XY + a * a * a * a;
    double sq = sqrt(Q);
    double fr = nn / (r2 * r) - 3.0 * Dnx * Dny / (r2 * r2 * r);
    double im = a * ((2.0 * Xnx * Yny - a * a * nn) / (Q * sq) -
                     3.0 * (XX * Yny - a * a * Xny) * (YY * Xnx - a * a * Ynx) / (Q * Q * sq));
    return (fr + im) / (4.0 * OR_PI);
}

/* Second-kind local BIE (Eq. bw55-bw59) on a flat (disk) patch.  For x and y
 * in the plane of S, which passes through the ball centre, X.n = Y.n = 0 and
 * (X - Y).n = 0, so dG/dn_x vanishes there: D = 0 and Eq. bw55 reads
 * q(x) = 2 b(x).  b is regularised with the constant solution (for u = 1,
 * q = 0: 0 = - int_Gamma K - p.f. int_S K), so at each collocation point
 *   q_i = - 2 sum_k W_k K(x_i, y_k) (U_k - g(x_i))
 *         - 2 p.v. int_S K(x_i, y) (g(y) - g(x_i)) ds_y,
 * K = d2G/dn_x dn_y, which on S is (1/4pi) (1/rho^3 - a^3 Q^{-3/2}).  The
 * linear Taylor term t(y) = grad_S g(x_i).(y - x_i) is taken out of the S
 * integral: its free-space part is exact, p.v. int_S (y - x)/rho^3 ds =
 * - oint_{dS} nu / rho dl (divergence theorem in the plane, nu the outward unit
 * normal of the disk's rim), by ng2 Gauss points on the rim; the rest
 * (g - g(x_i) - t) K and t times the image part are integrated in polar
 * coordinates about x_i, angle by ng2 Gauss points on [0, 2 pi], rho by ng2
 * on [0, rho_max(angle)].  grad_S g by central differences (h = 1e-5 a) along
 * t1, t2.  U: the hemisphere values at the nodes of or_gamma_nodes(p, nt, nph).
 * Returns -1 unless p is a disk patch. */
int or_second_kind_flat(const or_patch *p, const or_data *dat, int nt, int nph, int nr, int ns,
                        const double *U, int ng2, double *q)
{
    if (p->kind != 0) return -1;
    const int P = nt * nph, n = nr * ns;
    const double a = p->a;
    double *Yl = malloc(sizeof(double) * 3 * P), *W = malloc(sizeof(double) * P);
    double *Xl = malloc(sizeof(double) * 3 * n), *ar = malloc(sizeof(double) * n);
    double *xg = malloc(sizeof(double) * 3 * n);
    double *gx = malloc(sizeof(double) * ng2), *gw = malloc(sizeof(double) * ng2);
    or_gamma_nodes(p, nt, nph, Yl, NULL, W);
    or_panels(p, nr, ns, Xl, xg, NULL, ar, NULL);
    or_gauss_legendre(ng2, gx, gw);
    const double ez[3] = {0.0, 0.0, 1.0};
    for (int i = 0; i < n; ++i) {
        const double *X = Xl + 3 * i;
        double xglob[3];
        local_to_global(p, X, xglob);
        const double gxi = or_dirichlet(dat, xglob);
        /* Gamma term; the outward normal of the hemisphere is Y / a */
        double sg = 0.0;
        for (int k = 0; k < P; ++k) {
            const double *Y = Yl + 3 * k;
            double ny[3] = {Y[0] / a, Y[1] / a, Y[2] / a};
            sg += W[k] * or_green_dnn(a, X, ez, Y, ny) * (U[k] - gxi);
        }
        /* tangential gradient of the data at x_i */
        double grad[2];
        const double h = 1e-5 * a;
        for (int d = 0; d < 2; ++d) {
            double Lp[3] = {X[0], X[1], 0.0}, Lm[3] = {X[0], X[1], 0.0}, yp[3], ym[3];
            Lp[d] += h; Lm[d] -= h;
            local_to_global(p, Lp, yp);
            local_to_global(p, Lm, ym);
            grad[d] = (or_dirichlet(dat, yp) - or_dirichlet(dat, ym)) / (2.0 * h);
        }
        /* S term: polar coordinates about x_i, rho_max from |X + rho e| = a */
        double ss = 0.0;
        const double xx = X[0] * X[0] + X[1] * X[1];
        for (int j = 0; j < ng2; ++j) {
            const double ph = OR_PI * (gx[j] + 1.0), wph = OR_PI * gw[j];
            const double e[2] = {cos(ph), sin(ph)};
            const double xe = X[0] * e[0] + X[1] * e[1];
            const double rmax = -xe + sqrt(xe * xe + a * a - xx);
            for (int l = 0; l < ng2; ++l) {
                const double rho = 0.5 * rmax * (gx[l] + 1.0), w = wph * 0.5 * rmax * gw[l];
                const double L[3] = {X[0] + rho * e[0], X[1] + rho * e[1], 0.0};
                double yglob[3];
                local_to_global(p, L, yglob);
                const double t = rho * (grad[0] * e[0] + grad[1] * e[1]);
                const double XX = xx, YY = L[0] * L[0] + L[1] * L[1], XY = X[0] * L[0] + X[1] * L[1];
                const double Q = XX * YY - 2.0 * a * a * XY + a * a * a * a;
                const double img = a * a * a / (Q * sqrt(Q));
                /* (g - g(x) - t)(1/rho^3 - img) + t (- img), times the area element rho */
                ss += w * rho * ((or_dirichlet(dat, yglob) - gxi - t) * (1.0 / (rho * rho * rho) - img) - t * img);
            }
        }
        /* p.v. int_S (y - x)/rho^3 ds = - oint nu / rho dl over the rim |Y| = a */
        double pv[2] = {0.0, 0.0};
        for (int j = 0; j < ng2; ++j) {
            const double th = OR_PI * (gx[j] + 1.0), w = OR_PI * gw[j] * a;
            const double nu[2] = {cos(th), sin(th)};
            const double dy[2] = {a * nu[0] - X[0], a * nu[1] - X[1]};
            const double rr = sqrt(dy[0] * dy[0] + dy[1] * dy[1]);
            pv[0] -= w * nu[0] / rr;
            pv[1] -= w * nu[1] / rr;
        }
        ss += grad[0] * pv[0] + grad[1] * pv[1];
        q[i] = -2.0 * sg - 2.0 * ss / (4.0 * OR_PI);
    }
    free(Yl); free(W); free(Xl); free(ar); free(xg); free(gx); free(gw);
    return 0;
}

/* ============================================== adaptive panel quadrature */
/* Integrands over a patch panel, in the panel's (u, v) parameters. */
typedef struct {
    const or_patch *p;
    const or_data *dat;
    int kind;           /* 0: G(X,Y); 1: dG/dn_y(X,Y) (g(y) - g(x)); 2: G(X,Y) q_exact(y);
                           3: dG/dn_y(X,Y) g(y); 4: K(X,Y) (g(y) - l(Y)) + dG/dn_x(X,Y) a.n_y;
                           5: dG/dn_x(X,Y) (second kind, see or_second_kind) */
    double X[3];
    double gx;          /* g at the collocation point (kinds 1, 4) */
    double nx[3];       /* normal at X (kinds 4, 5) */
    double ga[3];       /* tangential gradient of g at X, l(Y) = gx + ga.(Y - X) (kind 4) */
    int piece;          /* wrapped patch: the piece the panel lies on */
} quad_ctx;

static double gl10_x[10], gl10_w[10];
static int gl10_ready = 0;

static void gl10_init(void)
{
    if (!gl10_ready) {
        or_gauss_legendre(10, gl10_x, gl10_w);
        gl10_ready = 1;
    }
}

static double integrand(const quad_ctx *c, double u, double v)
{
    double Y[3], nl[3], J;
    patch_point(c->p, c->piece, u, v, Y, nl, &J);
    if (c->kind == 0) return or_green(c->p->a, c->X, Y) * J;
    if (c->kind == 4 || c->kind == 5) {
        /* dG/dn_x(X, Y) = n_x . grad_X G(X, Y) = n_x . (grad_y G)(Y, X), G symmetric */
        double gX[3];
        or_green_grad_y(c->p->a, Y, c->X, gX);
        const double dnx = gX[0] * c->nx[0] + gX[1] * c->nx[1] + gX[2] * c->nx[2];
        if (c->kind == 5) return dnx * J;
        double y[3];
        local_to_global(c->p, Y, y);
        const double l = c->gx + c->ga[0] * (Y[0] - c->X[0]) + c->ga[1] * (Y[1] - c->X[1]) +
                         c->ga[2] * (Y[2] - c->X[2]);
        const double an = c->ga[0] * nl[0] + c->ga[1] * nl[1] + c->ga[2] * nl[2];
        return (or_green_dnn(c->p->a, c->X, c->nx, Y, nl) * (or_dirichlet(c->dat, y) - l) + dnx * an) * J;
    }
    double y[3];
    local_to_global(c->p, Y, y);
    if (c->kind == 1 || c->kind == 3) {
        double g[3];
        or_green_grad_y(c->p->a, c->X, Y, g);
        double dn = g[0] * nl[0] + g[1] * nl[1] + g[2] * nl[2];
        double gy = or_dirichlet(c->dat, y);
        return dn * (c->kind == 1 ? gy - c->gx : gy) * J;
    }
    double ng[3];
    for (int i = 0; i < 3; ++i) ng[i] = nl[0] * c->p->t1[i] + nl[1] * c->p->t2[i] + nl[2] * c->p->n[i];
    return or_green(c->p->a, c->X, Y) * or_neumann_exact(c->dat, y, ng) * J;
}

/* Globally adaptive 1-D integration (bisect the segment with the largest error
 * estimate until the summed estimate is below tol, or a segment budget is
 * spent).  Rule: 10-point Gauss-Legendre; error estimate of a segment =
 * |G10(whole) - G10(left) - G10(right)|, value = G10(left) + G10(right). */
typedef double (*fn1)(void *, double);

static double gl_apply(fn1 f, void *c, double a, double b)
{
    double h = 0.5 * (b - a), m = 0.5 * (a + b), s = 0.0;
    for (int i = 0; i < 10; ++i) s += gl10_w[i] * f(c, m + h * gl10_x[i]);
    return s * h;
}

#define OR_MAXSEG 160
static double gadapt(fn1 f, void *c, double a, double b, double tol)
{
    double sa[OR_MAXSEG], sb[OR_MAXSEG], sl[OR_MAXSEG], sr[OR_MAXSEG], se[OR_MAXSEG];
    double m = 0.5 * (a + b);
    double w = gl_apply(f, c, a, b);
    sa[0] = a; sb[0] = b;
    sl[0] = gl_apply(f, c, a, m); sr[0] = gl_apply(f, c, m, b);
    se[0] = fabs(sl[0] + sr[0] - w);
    int ns = 1;
    for (;;) {
        double tot = 0.0, mag = 0.0;
        int worst = 0;
        for (int i = 0; i < ns; ++i) {
            tot += se[i];
            mag += fabs(sl[i]) + fabs(sr[i]);
            if (se[i] > se[worst]) worst = i;
        }
        if (tot <= tol || tot <= 1e-15 * mag || ns + 1 >= OR_MAXSEG) break;
        /* split the worst segment into its two halves, each refined once */
        double a0 = sa[worst], b0 = sb[worst], m0 = 0.5 * (a0 + b0);
        double wl = sl[worst], wr = sr[worst];
        double q1 = 0.5 * (a0 + m0), q3 = 0.5 * (m0 + b0);
        double l1 = gl_apply(f, c, a0, q1), r1 = gl_apply(f, c, q1, m0);
        double l2 = gl_apply(f, c, m0, q3), r2 = gl_apply(f, c, q3, b0);
        sa[worst] = a0; sb[worst] = m0; sl[worst] = l1; sr[worst] = r1; se[worst] = fabs(l1 + r1 - wl);
        sa[ns] = m0; sb[ns] = b0; sl[ns] = l2; sr[ns] = r2; se[ns] = fabs(l2 + r2 - wr);
        ++ns;
    }
    double v = 0.0;
    for (int i = 0; i < ns; ++i) v += sl[i] + sr[i];
    return v;
}

/* Nested integration over a parameter box: outer over u, inner over v.  An
 * inner error d moves the outer integral by at most d (u1 - u0), so the inner
 * tolerance is a tenth of tol / (u1 - u0). */
typedef struct { const quad_ctx *q; double u, v0, v1, tol; } box_ctx;

static double box_inner(void *p, double v)
{
    box_ctx *b = (box_ctx *)p;
    return integrand(b->q, b->u, v);
}

static double box_outer(void *p, double u)
{
    box_ctx b = *(box_ctx *)p;
    b.u = u;
    return gadapt(box_inner, &b, b.v0, b.v1, b.tol);
}

static double rect_integral(const quad_ctx *c, double u0, double u1, double v0, double v1, double tol)
{
    box_ctx b = {c, 0.0, v0, v1, 0.1 * tol / (u1 - u0)};
    return gadapt(box_outer, &b, u0, u1, tol);
}

/* Triangle (S, A, B) in parameter space with the singular point at S, by the
 * Duffy map p(s,t) = S + s [(A - S) + t (B - A)], Jacobian s |det(A - S, B - A)|:
 * the factor s cancels the 1/r singularity at S (the local polar transform of
 * the self panel, Sec. 5.2).  Nested adaptive integration in (s, t). */
typedef struct {
    const quad_ctx *q;
    double S[2], E1[2], E2[2], det;
    double s, tol;
} duffy_ctx;

static double duffy_inner(void *p, double t)
{
    duffy_ctx *T = (duffy_ctx *)p;
    double u = T->S[0] + T->s * (T->E1[0] + t * T->E2[0]);
    double v = T->S[1] + T->s * (T->E1[1] + t * T->E2[1]);
    return integrand(T->q, u, v) * T->s * T->det;
}

static double duffy_outer(void *p, double s)
{
    duffy_ctx T = *(duffy_ctx *)p;
    T.s = s;
    return gadapt(duffy_inner, &T, 0.0, 1.0, T.tol);
}

static double duffy_triangle(const quad_ctx *c, const double S[2], const double A[2],
                             const double B[2], double tol)
{
    duffy_ctx T;
    T.q = c;
    T.S[0] = S[0]; T.S[1] = S[1];
    T.E1[0] = A[0] - S[0]; T.E1[1] = A[1] - S[1];
    T.E2[0] = B[0] - A[0]; T.E2[1] = B[1] - A[1];
    T.det = fabs(T.E1[0] * T.E2[1] - T.E1[1] * T.E2[0]);
    T.s = 0.0;
    T.tol = 0.1 * tol;
    if (T.det == 0.0) return 0.0;
    return gadapt(duffy_outer, &T, 0.0, 1.0, tol);
}

/* Exact integral (R9 reading: entries are the integrals themselves) of the
 * chosen integrand over one panel's parameter box.  If `sing` is given (the
 * collocation point lies on this panel) the box is cut into four triangles
 * from the singular parameter point and each is integrated through the Duffy
 * map.  `rtol` is relative to area / (4 pi max(distance, diameter)). */
static double panel_integral_ctx(quad_ctx c, const double prm[7], const double *sing, double rtol);

/* Gauss order per direction of the self-panel rule of the second-kind
 * integrands (see panel_integral_ctx).  Set before calls, not during them. */
static int sk_self_order = 20;

int or_set_sk_self_order(int n)
{
    int old = sk_self_order;
    if (n >= 4 && n <= 64) sk_self_order = n;
    return old;
}

double or_panel_integral(const or_patch *p, const or_data *dat, int kind, const double X[3],
                         const double prm[7], const double *sing, double rtol)
{
    quad_ctx c;
    memset(&c, 0, sizeof(c));
    c.p = p; c.dat = dat; c.kind = kind;
    c.X[0] = X[0]; c.X[1] = X[1]; c.X[2] = X[2];
    if (kind == 1) {
        double xg[3];
        local_to_global(p, X, xg);
        c.gx = or_dirichlet(dat, xg);
    }
    return panel_integral_ctx(c, prm, sing, rtol);
}

static double panel_integral_ctx(quad_ctx c, const double prm[7], const double *sing, double rtol)
{
    gl10_init();
    const or_patch *p = c.p;
    const double *X = c.X;
    double u0 = prm[0], u1 = prm[1], v0 = prm[2], v1 = prm[3];
    c.piece = (p->kind == 2) ? (int)prm[6] : 0;
    double Yc[3], nl[3], J;
    patch_point(p, c.piece, prm[4], prm[5], Yc, nl, &J);
    double d = sqrt((X[0] - Yc[0]) * (X[0] - Yc[0]) + (X[1] - Yc[1]) * (X[1] - Yc[1]) +
                    (X[2] - Yc[2]) * (X[2] - Yc[2]));
    double diam, area;
    if (p->kind == 2) {
        /* the largest distance between the panel's corners and edge midpoints,
         * and an upper bound of its area */
        double pts[8][3], nn[3], Jd;
        const double us[3] = {u0, 0.5 * (u0 + u1), u1}, vs[3] = {v0, 0.5 * (v0 + v1), v1};
        int m = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (!(i == 1 && j == 1)) patch_point(p, c.piece, us[i], vs[j], pts[m++], nn, &Jd);
        diam = 0.0;
        for (int i = 0; i < 8; ++i)
            for (int j = i + 1; j < 8; ++j)
                diam = fmax(diam, sqrt((pts[i][0] - pts[j][0]) * (pts[i][0] - pts[j][0]) +
                                       (pts[i][1] - pts[j][1]) * (pts[i][1] - pts[j][1]) +
                                       (pts[i][2] - pts[j][2]) * (pts[i][2] - pts[j][2])));
        area = diam * diam;
    } else if (p->kind == 0) {
        diam = (u1 - u0) + u1 * (v1 - v0);
        area = 0.5 * (u1 * u1 - u0 * u0) * (v1 - v0);
    } else {
        diam = fabs(p->R) * ((u1 - u0) + sin(u1) * (v1 - v0));
        area = p->R * p->R * (cos(u0) - cos(u1)) * (v1 - v0);
    }
    double tol = rtol * area / (4.0 * OR_PI * (d > diam ? d : diam));
    if (c.kind >= 1 && c.kind <= 3) {
        /* integrands that carry the data: relative to the integral of |f| (a
         * 10 x 10 Gauss estimate), since area / (4 pi d) is the size of G alone
         * and far from the data's own scale (a source far away makes g(y) -
         * g(x) small) */
        gl10_init();
        const double hu = 0.5 * (u1 - u0), hv = 0.5 * (v1 - v0);
        double mabs = 0.0;
        for (int i = 0; i < 10; ++i)
            for (int j = 0; j < 10; ++j)
                mabs += gl10_w[i] * gl10_w[j] *
                        fabs(integrand(&c, u0 + hu * (gl10_x[i] + 1.0), v0 + hv * (gl10_x[j] + 1.0)));
        tol = rtol * mabs * hu * hv;
    }
    if (!sing) return rect_integral(&c, u0, u1, v0, v1, tol);
    double S[2] = {sing[0], sing[1]};
    double cor[5][2] = {{u0, v0}, {u1, v0}, {u1, v1}, {u0, v1}, {u0, v0}};
    double s = 0.0;
    if (c.kind == 4 || c.kind == 5) {
        /* Second-kind integrands: bounded and smooth in the Duffy variables, but
         * next to the corner s = 0 rounding dominates them (g - l is O(r^2)
         * against g = O(1), divided by r^3; n_x.(x - y) is O(r^2) from
         * components of size r), so an adaptive split toward s = 0 would chase
         * rounding, and so does a high-order rule, whose first nodes sit close
         * to s = 0 (the rounding error of a node grows like 1/s^2).  A fixed
         * Gauss rule of order sk_self_order (default 20) per direction and
         * triangle; each triangle's far edge is cut into pieces no longer than
         * its height.  On cap and disk patches the orders 12 ... 24 agree to a
         * few 1e-12 of |q| (the smooth integrand has converged), while 40 and
         * 80 move q by 1e-11 ... 1e-10 (rounding at their first nodes). */
        const int NQ = sk_self_order;
        double gxs[64], gws[64];
        or_gauss_legendre(NQ, gxs, gws);
        double PS[3], nn[3], Jd;
        patch_point(p, c.piece, S[0], S[1], PS, nn, &Jd);
        for (int e = 0; e < 4; ++e) {
          /* the far edge cut into m pieces no longer than the triangle's height */
          double PA[3], PB[3];
          patch_point(p, c.piece, cor[e][0], cor[e][1], PA, nn, &Jd);
          patch_point(p, c.piece, cor[e + 1][0], cor[e + 1][1], PB, nn, &Jd);
          double ab[3] = {PB[0] - PA[0], PB[1] - PA[1], PB[2] - PA[2]};
          double as[3] = {PS[0] - PA[0], PS[1] - PA[1], PS[2] - PA[2]};
          double cr[3];
          cross3(ab, as, cr);
          double L = sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
          double hh = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]) / (L > 0 ? L : 1.0);
          int m = (int)ceil(L / (hh > 0 ? hh : 1.0));
          if (m < 1) m = 1;
          if (m > 64) m = 64;
          for (int piece = 0; piece < m; ++piece) {
            double A0[2] = {cor[e][0] + (cor[e + 1][0] - cor[e][0]) * piece / m,
                            cor[e][1] + (cor[e + 1][1] - cor[e][1]) * piece / m};
            double B0[2] = {cor[e][0] + (cor[e + 1][0] - cor[e][0]) * (piece + 1) / m,
                            cor[e][1] + (cor[e + 1][1] - cor[e][1]) * (piece + 1) / m};
            double E1[2] = {A0[0] - S[0], A0[1] - S[1]};
            double E2[2] = {B0[0] - A0[0], B0[1] - A0[1]};
            double det = fabs(E1[0] * E2[1] - E1[1] * E2[0]);
            if (det == 0.0) continue;
            for (int i = 0; i < NQ; ++i) {
                double sv = 0.5 * (gxs[i] + 1.0);
                for (int j = 0; j < NQ; ++j) {
                    double tv = 0.5 * (gxs[j] + 1.0);
                    double u = S[0] + sv * (E1[0] + tv * E2[0]);
                    double v = S[1] + sv * (E1[1] + tv * E2[1]);
                    s += 0.25 * gws[i] * gws[j] * integrand(&c, u, v) * sv * det;
                }
            }
          }
        }
        return s;
    }
    for (int e = 0; e < 4; ++e) s += duffy_triangle(&c, S, cor[e], cor[e + 1], 0.25 * tol);
    return s;
}

/* ================================================================ assembly */
/* Collocation of the first-kind local BIE, Eq. bw49-bw51, at the panel
 * collocation points x_i with piecewise-constant Neumann data on the panels:
 *   A_ij = int_{panel j} G(x_i, y) ds_y.
 * The right side b of Eq. bw51 is taken with the constant solution subtracted,
 * as the paper does for its single-point formula (Sec. 3, Eq. bw61-bw68): for
 * u = 1 (zero Neumann data) Eq. bw51 reads 0 = 1/2 + p.v. int_S dG/dn_y +
 * int_Gamma dG/dn_y, and subtracting g(x_i) times that identity gives
 *   b_i = int_S dG/dn_y(x_i, y) (g(y) - g(x_i)) ds_y
 *         - sum_k W_k P(x_i, y_k) (U_k - g(x_i)),
 * where the Gamma integral of dG/dn_y u is minus the Poisson-kernel quadrature
 * over the hemisphere nodes and U_k are the walk estimates of u there.  On a
 * plane through c both terms of dG/dn_y vanish, so the S integral is zero for
 * flat patches. */
int or_assemble(const or_patch *p, const or_data *dat, int nr, int ns, int nt, int nph,
                const double *U, double rtol, double *A, double *b)
{
    int n = nr * ns, P = nt * nph;
    double *Xl = malloc(sizeof(double) * 3 * n), *xg = malloc(sizeof(double) * 3 * n);
    double *ar = malloc(sizeof(double) * n), *prm = malloc(sizeof(double) * OR_PRM * n);
    double *Yl = malloc(sizeof(double) * 3 * P), *W = malloc(sizeof(double) * P);
    if (or_panels(p, nr, ns, Xl, xg, NULL, ar, prm) != 0) {
        free(Xl); free(xg); free(ar); free(prm); free(Yl); free(W);
        return -1;
    }
    or_gamma_nodes(p, nt, nph, Yl, NULL, W);
    gl10_init();
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; ++i) {
        double gxi = or_dirichlet(dat, xg + 3 * i);
        double bi = 0.0;
        for (int j = 0; j < n; ++j) {
            const double *sing = (i == j) ? prm + OR_PRM * i + 4 : NULL;
            A[(int64_t)i * n + j] = or_panel_integral(p, dat, 0, Xl + 3 * i, prm + OR_PRM * j, sing, rtol);
            /* dG/dn_y vanishes on a plane through c (disk patches, and the
             * wrapped patch's first piece, where it is integrated anyway) */
            if (p->kind == 1 || p->kind == 2)
                bi += or_panel_integral(p, dat, 1, Xl + 3 * i, prm + OR_PRM * j, sing, rtol);
        }
        for (int k = 0; k < P; ++k)
            bi -= W[k] * or_poisson(p->a, Xl + 3 * i, Yl + 3 * k) * (U[k] - gxi);
        b[i] = bi;
    }
    free(Xl); free(xg); free(ar); free(prm); free(Yl); free(W);
    return 0;
}

/* ============================================= second kind, any patch */
/* Second-kind local BIE (Eq. bw55-bw59) on a disk or cap patch, collocated at
 * the panel collocation points with piecewise-constant Neumann data:
 *   (1/2) q_i - sum_j D_ij q_j = b_i,   D_ij = int_{panel j} dG/dn_x(x_i, y) ds_y.
 * The Hadamard finite part in b (Eq. bw59) is regularised with the harmonic
 * function l_i(y) = g(x_i) + a_i.(y - x_i), a_i the tangential gradient of g
 * at x_i (central differences, h = 1e-5 a, along the two unit tangents of the
 * patch there): Eq. bw55 holds for l_i itself, whose Neumann data is a_i.n_y
 * and a_i.n_x = 0, so
 *   p.f. int_S K l_i = - int_Gamma K l_i + D[a_i.n](x_i),
 * and
 *   b_i = - sum_k W_k K(x_i, y_k) (U_k - l_i(y_k))
 *         - int_S [ K(x_i, y) (g(y) - l_i(y)) + dG/dn_x(x_i, y) a_i.n_y ] ds_y,
 * K = d2G/dn_x dn_y; g - l_i = O(|y - x_i|^2) on S, so every integrand is
 * O(1/|y - x_i|) and the self panel goes through the Duffy map.  Entries by
 * the adaptive rules of or_panel_integral (relative tolerance rtol).  A (n x n,
 * row-major) and b are written when not NULL; q receives the solution.  U: the
 * hemisphere values at the nodes of or_gamma_nodes(p, nt, nph).  Returns the
 * status of the LU solve. */
int or_lu_solve(int n, double *A, double *b, double *x);

int or_second_kind(const or_patch *p, const or_data *dat, int nt, int nph, int nr, int ns, const double *U,
                   double rtol, double *A_out, double *b_out, double *q)
{
    if (p->kind == 2) return -2;   /* the second kind is written for disk and cap patches */
    const int n = nr * ns, P = nt * nph;
    const double a = p->a;
    double *Xl = malloc(sizeof(double) * 3 * n), *xg = malloc(sizeof(double) * 3 * n);
    double *ar = malloc(sizeof(double) * n), *prm = malloc(sizeof(double) * OR_PRM * n);
    double *Yl = malloc(sizeof(double) * 3 * P), *W = malloc(sizeof(double) * P);
    double *A = malloc(sizeof(double) * (size_t)n * n), *b = malloc(sizeof(double) * n);
    or_panels(p, nr, ns, Xl, xg, NULL, ar, prm);
    or_gamma_nodes(p, nt, nph, Yl, NULL, W);
    gl10_init();
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; ++i) {
        const double *X = Xl + 3 * i;
        double Yc[3], nx[3], J;
        patch_point(p, 0, prm[OR_PRM * i + 4], prm[OR_PRM * i + 5], Yc, nx, &J);
        /* unit tangents at the collocation point: along u and along v */
        const double uc = prm[OR_PRM * i + 4], vc = prm[OR_PRM * i + 5];
        double e1[3], e2[3] = {-sin(vc), cos(vc), 0.0};
        if (p->kind == 0) { e1[0] = cos(vc); e1[1] = sin(vc); e1[2] = 0.0; }
        else { e1[0] = cos(uc) * cos(vc); e1[1] = cos(uc) * sin(vc); e1[2] = -sin(uc); }
        const double h = 1e-5 * a;
        double ga[3] = {0.0, 0.0, 0.0};
        const double *ev[2] = {e1, e2};
        for (int d = 0; d < 2; ++d) {
            double Lp[3], Lm[3], yp[3], ym[3];
            for (int k = 0; k < 3; ++k) { Lp[k] = X[k] + h * ev[d][k]; Lm[k] = X[k] - h * ev[d][k]; }
            local_to_global(p, Lp, yp);
            local_to_global(p, Lm, ym);
            const double dg = (or_dirichlet(dat, yp) - or_dirichlet(dat, ym)) / (2.0 * h);
            for (int k = 0; k < 3; ++k) ga[k] += dg * ev[d][k];
        }
        quad_ctx c;
        memset(&c, 0, sizeof(c));
        c.p = p; c.dat = dat;
        for (int k = 0; k < 3; ++k) { c.X[k] = X[k]; c.nx[k] = nx[k]; c.ga[k] = ga[k]; }
        c.gx = or_dirichlet(dat, xg + 3 * i);
        double bi = 0.0;
        for (int j = 0; j < n; ++j) {
            const double *sing = (i == j) ? prm + OR_PRM * i + 4 : NULL;
            c.kind = 5;
            const double dij = panel_integral_ctx(c, prm + OR_PRM * j, sing, rtol);
            A[(int64_t)i * n + j] = (i == j ? 0.5 : 0.0) - dij;
            c.kind = 4;
            bi -= panel_integral_ctx(c, prm + OR_PRM * j, sing, rtol);
        }
        for (int k = 0; k < P; ++k) {
            const double *Y = Yl + 3 * k;
            const double ny[3] = {Y[0] / a, Y[1] / a, Y[2] / a};
            const double l = c.gx + ga[0] * (Y[0] - X[0]) + ga[1] * (Y[1] - X[1]) + ga[2] * (Y[2] - X[2]);
            bi -= W[k] * or_green_dnn(a, X, nx, Y, ny) * (U[k] - l);
        }
        b[i] = bi;
    }
    if (A_out) memcpy(A_out, A, sizeof(double) * (size_t)n * n);
    if (b_out) memcpy(b_out, b, sizeof(double) * n);
    int st = or_lu_solve(n, A, b, q);
    free(Xl); free(xg); free(ar); free(prm); free(Yl); free(W); free(A); free(b);
    return st;
}

/* ======================================================================= LU */
/* Dense LU with partial pivoting (pivot = first row of maximal |a|), then
 * forward and back substitution.  A (row-major n x n) and b are overwritten.
 * Returns 0, or k+1 if the k-th pivot is exactly zero. */
int or_lu_solve(int n, double *A, double *b, double *x)
{
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = fabs(A[(int64_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = fabs(A[(int64_t)i * n + k]);
            if (v > best) { best = v; piv = i; }
        }
        if (best == 0.0) return k + 1;
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[(int64_t)k * n + j];
                A[(int64_t)k * n + j] = A[(int64_t)piv * n + j];
                A[(int64_t)piv * n + j] = t;
            }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double l = A[(int64_t)i * n + k] / A[(int64_t)k * n + k];
            A[(int64_t)i * n + k] = l;
            for (int j = k + 1; j < n; ++j) A[(int64_t)i * n + j] -= l * A[(int64_t)k * n + j];
            b[i] -= l * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[(int64_t)i * n + j] * x[j];
        x[i] = s / A[(int64_t)i * n + i];
    }
    return 0;
}

/* =========================================================== full patch */
/* Steps 1 and 2 of the BIE-WOS algorithm (Sec. 4) for one patch: walks at the
 * hemisphere nodes, then assembly and solve.  If U_in is given the walks are
 * skipped and U_in is used. */
int or_solve_patch(const or_geom *g, const or_data *dat, const double c[3], double a, int nt,
                   int nph, int nr, int ns, int64_t walks, uint32_t patch_id,
                   const or_wos_opts *o, const double *U_in, double rtol, double *U_out,
                   double *SE_out, uint64_t *steps_out, double *q_out)
{
    or_patch p;
    if (or_patch_frame(g, c, a, &p) != 0) return -1;
    int P = nt * nph, n = nr * ns;
    double *U = malloc(sizeof(double) * P);
    if (U_in) {
        memcpy(U, U_in, sizeof(double) * P);
        if (steps_out) *steps_out = 0;
    } else {
        double *y = malloc(sizeof(double) * 3 * P), *W = malloc(sizeof(double) * P);
        double *s1 = malloc(sizeof(double) * P), *s2 = malloc(sizeof(double) * P);
        uint64_t *st = malloc(sizeof(uint64_t) * P), *cp = malloc(sizeof(uint64_t) * P);
        uint32_t *pt = malloc(sizeof(uint32_t) * P), *pa = malloc(sizeof(uint32_t) * P);
        int64_t *wk = malloc(sizeof(int64_t) * P);
        or_gamma_nodes(&p, nt, nph, NULL, y, W);
        for (int k = 0; k < P; ++k) { pt[k] = (uint32_t)k; pa[k] = patch_id; wk[k] = walks; }
        or_wos_points(g, dat, P, y, pt, pa, wk, o, s1, s2, st, cp);
        uint64_t tot = 0;
        for (int k = 0; k < P; ++k) {
            double N = (double)(walks - (int64_t)cp[k]);
            U[k] = s1[k] / N;
            double var = (s2[k] - N * U[k] * U[k]) / (N * (N - 1.0));
            if (SE_out) SE_out[k] = sqrt(var > 0 ? var : 0.0);
            tot += st[k];
        }
        if (steps_out) *steps_out = tot;
        free(y); free(W); free(s1); free(s2); free(st); free(cp); free(pt); free(pa); free(wk);
    }
    if (U_out) memcpy(U_out, U, sizeof(double) * P);
    double *A = malloc(sizeof(double) * n * n), *b = malloc(sizeof(double) * n);
    int rc = or_assemble(&p, dat, nr, ns, nt, nph, U, rtol, A, b);
    if (rc == 0) rc = or_lu_solve(n, A, b, q_out);
    free(A); free(b); free(U);
    return rc;
}

/* ======================================================= single point */
/* Neumann data at one point x of a flat boundary piece, Sec. 4.1 (Eq. bw64):
 *   q(x) = Sigma1' + Sigma2',
 *   Sigma1' = - int_Gamma d2g/dn_x dn_y (u(y) - g(x)) ds_y        (Eq. bw65)
 *           ~ - sum_ij W_ij (3 cos th_i / (2 pi a^3)) (U_ij - g(x))  (Eq. bw83, bw85)
 * with the hemisphere nodes and weights of or_gamma_nodes (theta_max = pi/2), the
 * normal second derivative of the half-ball Green's function on Gamma being
 * 3 cos th / (2 pi a^3); U_ij are WOS estimates (Eq. bw87) or given values;
 *   Sigma2' = -(1/2pi) int_{S_a minus disk(x, delta)} (1/rho^3 - 1/a^3) (g(y) - g(x)) ds_y
 * (Eq. bw68 with the small disk of Eq. bw73-bw82 removed, an O(delta) error),
 * by the ng2 x ng2 Gauss rule in polar coordinates about x: rho in [delta, a],
 * angle in [0, 2 pi], ds = rho drho dangle.
 * out: Sigma1', Sigma2', q, standard error of Sigma1'.  U_in (ng1^2 values) or NULL
 * to run `walks` walks per node (node k = i*ng1 + j is the RNG point id, `patch`
 * the RNG patch id).  U_out (ng1^2) receives the node values if not NULL.
 * Returns 0, or -1 if x is not on a supported flat piece. */
int or_single_point(const or_geom *g, const or_data *dat, const double x[3], double a, int ng1,
                    int ng2, double delta, int64_t walks, uint32_t patch, const or_wos_opts *o,
                    const double *U_in, double out[4], double *U_out)
{
    or_patch p;
    if (or_patch_frame(g, x, a, &p) != 0 || p.kind != 0) return -1;
    const int nn = ng1 * ng1;
    double *Yl = malloc(sizeof(double) * 3 * nn), *yg = malloc(sizeof(double) * 3 * nn);
    double *W = malloc(sizeof(double) * nn), *U = malloc(sizeof(double) * nn);
    double *SE = malloc(sizeof(double) * nn);
    or_gamma_nodes(&p, ng1, ng1, Yl, yg, W);
    if (U_in) {
        for (int k = 0; k < nn; ++k) { U[k] = U_in[k]; SE[k] = 0.0; }
    } else {
#pragma omp parallel for schedule(dynamic, 1)
        for (int k = 0; k < nn; ++k) {
            double s1, s2;
            uint64_t st, cap;
            or_wos_point(g, dat, yg + 3 * k, (uint32_t)k, patch, 0, walks, o, &s1, &s2, &st, &cap);
            double N = (double)(walks - (int64_t)cap);
            U[k] = s1 / N;
            double var = (s2 - N * U[k] * U[k]) / (N * (N - 1.0));
            SE[k] = sqrt(fmax(var, 0.0));
        }
    }
    const double gx = or_dirichlet(dat, x);
    double s1 = 0.0, v1 = 0.0;
    for (int k = 0; k < nn; ++k) {
        double cth = -Yl[3 * k + 2] / a;
        double wk = W[k] * 3.0 * cth / (2.0 * OR_PI * a * a * a);
        s1 -= wk * (U[k] - gx);
        v1 += wk * wk * SE[k] * SE[k];
    }
    double *xr = malloc(sizeof(double) * ng2), *wr = malloc(sizeof(double) * ng2);
    or_gauss_legendre(ng2, xr, wr);
    double s2 = 0.0;
    for (int i = 0; i < ng2; ++i) {
        double rho = delta + 0.5 * (a - delta) * (xr[i] + 1.0);
        double wrho = 0.5 * (a - delta) * wr[i];
        for (int j = 0; j < ng2; ++j) {
            double ang = OR_PI * (xr[j] + 1.0);
            double L[3] = {rho * cos(ang), rho * sin(ang), 0.0};
            double y[3];
            local_to_global(&p, L, y);
            s2 += wrho * OR_PI * wr[j] * rho * (1.0 / (rho * rho * rho) - 1.0 / (a * a * a)) *
                  (or_dirichlet(dat, y) - gx);
        }
    }
    s2 *= -1.0 / (2.0 * OR_PI);
    out[0] = s1; out[1] = s2; out[2] = s1 + s2; out[3] = sqrt(v1);
    if (U_out)
        for (int k = 0; k < nn; ++k) U_out[k] = U[k];
    free(Yl); free(yg); free(W); free(U); free(SE); free(xr); free(wr);
    return 0;
}

/* ============================================================== potential */
/* Integral representation Eq. bw03 with G0 = 1/(4pi|x-y|) (Eq. bw05) and the
 * panel-midpoint rule:
 *   u(t) = sum_p A_p [ q_p / (4pi|t-y_p|) - g_p n_p.(t-y_p) / (4pi|t-y_p|^3) ]. */
void or_potential(int64_t np, const double *y, const double *nrm, const double *area,
                  const double *q, const double *g, int64_t nt, const double *t, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nt; ++i) {
        double s = 0.0;
        for (int64_t p = 0; p < np; ++p) {
            double d[3] = {t[3 * i] - y[3 * p], t[3 * i + 1] - y[3 * p + 1], t[3 * i + 2] - y[3 * p + 2]};
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double dn = d[0] * nrm[3 * p] + d[1] * nrm[3 * p + 1] + d[2] * nrm[3 * p + 2];
            s += area[p] * (q[p] / (4.0 * OR_PI * r) - g[p] * dn / (4.0 * OR_PI * r * r * r));
        }
        out[i] = s;
    }
}

/* Majorants of the sum above, per target: b0 = sum_p |A_p q_p| / (4pi|t-y_p|)
 * and b1 = sum_p |A_p g_p| / (4pi|t-y_p|^2) (the charge and dipole magnitudes
 * over the first and second power of the distance).  They scale the error
 * bound of an approximate evaluation (a multipole expansion) of or_potential. */
void or_potential_majorants(int64_t np, const double *y, const double *area, const double *q,
                            const double *g, int64_t nt, const double *t, double *b0, double *b1)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nt; ++i) {
        double s0 = 0.0, s1 = 0.0;
        for (int64_t p = 0; p < np; ++p) {
            double d[3] = {t[3 * i] - y[3 * p], t[3 * i + 1] - y[3 * p + 1], t[3 * i + 2] - y[3 * p + 2]};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double r = sqrt(r2);
            s0 += fabs(area[p] * q[p]) / (4.0 * OR_PI * r);
            s1 += fabs(area[p] * g[p]) / (4.0 * OR_PI * r2);
        }
        b0[i] = s0;
        b1[i] = s1;
    }
}

/* Panel ownership for the overlapping-patch cover (Sec. 6): panel of patch p is
 * kept iff the patch centre nearest to its collocation point is p's (lowest
 * index on ties).  keep[i] = 1 / 0. */
void or_owned(int64_t npan, const double *x, const int64_t *owner_patch, int64_t ncent,
              const double *cent, uint8_t *keep)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npan; ++i) {
        int64_t best = -1;
        double bd = INFINITY;
        for (int64_t c = 0; c < ncent; ++c) {
            double d[3] = {x[3 * i] - cent[3 * c], x[3 * i + 1] - cent[3 * c + 1], x[3 * i + 2] - cent[3 * c + 2]};
            double r = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r < bd) { bd = r; best = c; }
        }
        keep[i] = (best == owner_patch[i]) ? 1 : 0;
    }
}

/* Host threads of the OpenMP loops (timing the oracle on one core). */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
