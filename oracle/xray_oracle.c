/*
 * X-ray transform oracle: a plain, slow, double-precision CPU implementation.
 *
 * TEST INFRASTRUCTURE ONLY.  It is called by the test-suite, by the package's smoke check
 * and by the benchmark's CPU-baseline / reference leg.  The CUDA library never links or
 * calls it, and it shares no code, header, table or helper with the CUDA library.
 *
 * It follows Chen, Wang, Bajaj, Oktem, "A Fast and Adaptive Algorithm to Compute the
 * X-ray Transform", step by step:
 *
 *   1. ray parameters from the scan: eq. 2Dparalleltofan (equiangular fan),
 *      eq. 2Dparalleltofan_2 (equispaced fan), eq. equiangular_cone_beam,
 *      eq. equispaced_cone_beam, eq. Helical_cone_beam_equiangular,
 *      eq. Helical_cone_beam_equispaced; a ray list gives each ray's parallel-beam
 *      parameters directly (Section 4.3, Adaptability);
 *   2. the ray symmetries that bring a 2D ray to phi in [0, pi) (Section 2.2.1) and a 3D ray
 *      to (phi1, phi2) in [0, 2pi) x [0, pi/2] (Section 3.2.1);
 *   3. the ray point and direction: eq. direction_normal (2D), eq. 3Dparallel_direction,
 *      eq. theta_1, eq. theta_2 (3D);
 *   4. Case 1 (oblique ray): loop over the driving index i as in Algorithm 1 / Algorithm 2;
 *      C_x of eq. C_xC_y / C_xC_yC_z; the open range of valid j from eq. restriction_j /
 *      restriction_j_3D; the open range of valid k from eq. restriction_k_3D_1; C_low, C_up
 *      of eq. conditions_2D_1 / conditions_3D_1 and the length C_up - C_low of
 *      eq. range_length / range_length_3D for every candidate with C_low < C_up;
 *   5. Case 2 of Section 2.2.1 (phi = 0) and its Remark (phi = pi/2); Case 2 of Section
 *      3.2.1 (ray in a coordinate plane) and its Remark; Cases 3 and 4 (ray parallel to an
 *      axis): the closed index ranges printed there;
 *   6. the ambiguity rule of Section 4.1: when a closed range holds two indices, the unit
 *      with the bigger 1D index is taken.
 *
 * Readings where the paper is silent (each listed with its reason in the design notes):
 *   R1  1D index I = (k*ny + j)*nx + i (the printed "j*N_y + i" agrees with every table only
 *       because the examples are square).
 *   R2  x grows with i, y falls with j, z falls with k (the unit supports of eq.
 *       pixel_basis_function / voxel_basis_function).
 *   R3  "slight changes" for the other quadrants (Remark cases_2D, Remark case1_3D): the
 *       t-interval of a unit along an axis is [min(C, C'), max(C, C')], C the printed
 *       formula and C' its printed other end (C_x + 1/cos, C_y - 1/sin, ...); the open range
 *       of valid indices becomes (min(e1, e2) - 1, max(e1, e2)) with e1, e2 the printed
 *       bounds (C_1 and C_1 - tan(phi), ...).  In Case 1 this is the printed range; for
 *       phi in (pi/2, pi) it reproduces the hand computation of Test suite 2.
 *   R4  scale and centre (Section 4.2): the ray is expressed in the frame
 *       x' = (x - c_x)/d_x (same for y, z) with direction theta_a/d_a, so the printed
 *       formulas hold unchanged and t stays a physical length.
 *   R5  a horizontal oblique 3D ray (phi2 = 0, phi1 not a multiple of pi/2) is handled like
 *       Case 2 with the roles of y and z exchanged: k from a closed range, then the 2D
 *       Case 1 in the (x, y) plane.
 *   R6  detector samples are bin centres; a flat detector at distance sdd from the source
 *       maps to the paper's (t, h) on the plane through the origin by t = u*sod/sdd.
 *   R7  direction components with |cos|, |sin| < 1e-12 are exactly zero (an angle that is
 *       a multiple of pi/2 up to rounding).
 *   R15 the attenuated transform integrates the attenuation along +theta of the ray's own
 *       parameters (the side the ray runs towards).
 *
 * Precision: binary64, no FMA contraction (build with -ffp-contract=off).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { K_PAR2D = 0, K_FAN2D = 1, K_FAN2D_ARC = 2, K_PAR3D = 3, K_CONE = 4, K_CONE_ARC = 5,
       K_HELIX = 6, K_HELIX_ARC = 7, K_RAYS2D = 8, K_RAYS3D = 9 };

typedef struct {
    int kind;
    int nx, ny, nz;
    double dx, dy, dz;
    double cx, cy, cz;
    int n_views, n_rows, n_cols;
    const double *angles; /* n_views, or 2*n_views (phi1, phi2) for parallel 3D; ray lists:
                             (s, phi) per ray (2D) or (s1, s2, phi1, phi2) per ray (3D) */
    const double *src_z;  /* n_views for helical kinds, else NULL */
    double du, dv, u0, v0;
    double sod, sdd;
} orc_geom;

static int is3d(const orc_geom *g) { return g->kind >= K_PAR3D && g->kind != K_RAYS2D; }

/* ---------------------------------------------------------------------------------------
 * Unit lists and the optional trace of intermediate quantities
 * ------------------------------------------------------------------------------------- */

typedef struct {
    long *idx;
    double *len;
    int n, cap;
    int overflow;
    double *trace; /* records of 8 doubles, or NULL */
    int n_trace, cap_trace;
} orc_list;

static void push_unit(orc_list *L, long I, double l)
{
    if (L->n < L->cap) {
        L->idx[L->n] = I;
        L->len[L->n] = l;
        L->n++;
    } else {
        L->overflow = 1;
    }
}

static void push_trace(orc_list *L, double a0, double a1, double a2, double a3, double a4,
                       double a5, double a6, double a7)
{
    if (!L->trace || L->n_trace >= L->cap_trace) return;
    double *r = L->trace + 8 * (size_t)L->n_trace++;
    r[0] = a0; r[1] = a1; r[2] = a2; r[3] = a3; r[4] = a4; r[5] = a5; r[6] = a6; r[7] = a7;
}

/* smallest integer strictly above x / largest integer strictly below x */
static long int_above(double x) { return (long)floor(x) + 1; }
static long int_below(double x) { return (long)ceil(x) - 1; }

/* Closed range [lo, hi] of one index, clipped to [0, n-1]; the ambiguity rule of
 * Section 4.1 keeps the bigger index.  Returns -1 when the range is empty. */
static long closed_range_pick(double lo, double hi, long n)
{
    long a = (long)ceil(lo), b = (long)floor(hi);
    if (a < 0) a = 0;
    if (b > n - 1) b = n - 1;
    return (a <= b) ? b : -1;
}

/* ---------------------------------------------------------------------------------------
 * Case 1 in a plane (Section 2.2.1, Algorithm 1).  Axis P is oriented like x (its unit n
 * covers [n - NP/2, n - NP/2 + 1]), axis Q like y (unit n covers [NQ/2 - n - 1, NQ/2 - n]).
 * pP, pQ: the ray point; tP, tQ: the direction (both nonzero, any sign; R3).
 * The 1D index of unit (a, b) is base + a*sa + b*sb.
 * ------------------------------------------------------------------------------------- */
static void case1_plane(long NP, double pP, double tP, long NQ, double pQ, double tQ,
                        long base, long sa, long sb, orc_list *L)
{
    const double tan_phi = tQ / tP;
    for (long a = 0; a < NP; ++a) {
        /* eq. C_xC_y: C_x, and the other end of the x-interval (eq. condition_nonzero_t) */
        const double Cx = (a - NP / 2.0 - pP) / tP;
        const double Cx_other = Cx + 1.0 / tP;
        /* eq. restriction_j: C_1 - tan(phi) - 1 < j < C_1 (R3 for the other signs) */
        const double C1 = NQ / 2.0 - pQ - Cx * tQ;
        const double e1 = C1, e2 = C1 - tan_phi;
        const double lo = fmin(e1, e2) - 1.0, hi = fmax(e1, e2);
        push_trace(L, 0.0, (double)a, Cx, C1, lo, hi, 0.0, 0.0);
        long b0 = int_above(lo), b1 = int_below(hi);
        if (b0 < 0) b0 = 0;
        if (b1 > NQ - 1) b1 = NQ - 1;
        for (long b = b0; b <= b1; ++b) {
            /* eq. C_xC_y: C_y, and the other end of the y-interval */
            const double Cy = (NQ / 2.0 - b - pQ) / tQ;
            const double Cy_other = Cy - 1.0 / tQ;
            /* eq. conditions_2D_1 */
            const double Clow = fmax(fmin(Cx, Cx_other), fmin(Cy, Cy_other));
            const double Cup = fmin(fmax(Cx, Cx_other), fmax(Cy, Cy_other));
            push_trace(L, 1.0, (double)a, (double)b, Cy, 0.0, 0.0, Clow, Cup);
            if (Clow < Cup) push_unit(L, base + a * sa + b * sb, Cup - Clow); /* eq. range_length */
        }
    }
}

/* ---------------------------------------------------------------------------------------
 * Case 1 in space (Section 3.2.1, Algorithm 2).  x oriented up with i, y and z down with j, k.
 * ------------------------------------------------------------------------------------- */
static void case1_space(const orc_geom *g, double px, double py, double pz, double tx, double ty,
                        double tz, orc_list *L)
{
    const long Nx = g->nx, Ny = g->ny, Nz = g->nz;
    const double tan1 = ty / tx; /* tan(phi1) */
    const double tz_tx = tz / tx; /* tan(phi2)/cos(phi1) */
    const double tz_ty = tz / ty; /* tan(phi2)/sin(phi1) */
    for (long i = 0; i < Nx; ++i) {
        /* eq. C_xC_yC_z: C_x, and the other end of the x-interval (eq. condition_nonzero_t_3D) */
        const double Cx = (i - Nx / 2.0 - px) / tx;
        const double Cx_other = Cx + 1.0 / tx;
        /* eq. restriction_j_3D */
        const double C1 = Ny / 2.0 - py - Cx * ty;
        const double jlo = fmin(C1, C1 - tan1) - 1.0, jhi = fmax(C1, C1 - tan1);
        /* eq. restriction_k_3D_1, first line */
        const double C2 = Nz / 2.0 - pz - Cx * tz;
        const double k2lo = fmin(C2, C2 - tz_tx) - 1.0, k2hi = fmax(C2, C2 - tz_tx);
        push_trace(L, 0.0, (double)i, Cx, C1, jlo, jhi, C2, 0.0);
        long j0 = int_above(jlo), j1 = int_below(jhi);
        if (j0 < 0) j0 = 0;
        if (j1 > Ny - 1) j1 = Ny - 1;
        for (long j = j0; j <= j1; ++j) {
            const double Cy = (Ny / 2.0 - j - py) / ty;
            const double Cy_other = Cy - 1.0 / ty;
            /* eq. restriction_k_3D_1, second line */
            const double C3 = Nz / 2.0 - pz - Cy * tz;
            const double k3lo = fmin(C3, C3 + tz_ty) - 1.0, k3hi = fmax(C3, C3 + tz_ty);
            const double klo = fmax(k2lo, k3lo), khi = fmin(k2hi, k3hi);
            push_trace(L, 1.0, (double)i, (double)j, Cy, klo, khi, C3, 0.0);
            long k0 = int_above(klo), k1 = int_below(khi);
            if (k0 < 0) k0 = 0;
            if (k1 > Nz - 1) k1 = Nz - 1;
            for (long k = k0; k <= k1; ++k) {
                const double Cz = (Nz / 2.0 - k - pz) / tz;
                const double Cz_other = Cz - 1.0 / tz;
                /* eq. conditions_3D_1 */
                const double Clow = fmax(fmax(fmin(Cx, Cx_other), fmin(Cy, Cy_other)),
                                         fmin(Cz, Cz_other));
                const double Cup = fmin(fmin(fmax(Cx, Cx_other), fmax(Cy, Cy_other)),
                                        fmax(Cz, Cz_other));
                push_trace(L, 2.0, (double)i, (double)j, (double)k, Cz, Clow, Cup, 0.0);
                if (Clow < Cup)
                    push_unit(L, (k * Ny + j) * Nx + i, Cup - Clow); /* eq. range_length_3D */
            }
        }
    }
}

/* Closed ranges of Case 2 (2D), Cases 2-4 (3D): x-like axis / y-like axis (R2). */
static long pick_x(double p, long N) { return closed_range_pick(p + N / 2.0 - 1.0, p + N / 2.0, N); }
static long pick_y(double p, long N) { return closed_range_pick(N / 2.0 - p - 1.0, N / 2.0 - p, N); }

/* 2D: ray point (px, py) and direction (tx, ty) in the scaled frame (R4). */
static void units_2d(const orc_geom *g, double px, double py, double tx, double ty, orc_list *L)
{
    const long Nx = g->nx, Ny = g->ny;
    if (ty == 0.0 && tx == 0.0) return;
    if (ty == 0.0) {
        /* Case 2 (phi = 0): unit length for j in [N_y/2 - s - 1, N_y/2 - s] */
        long j = pick_y(py, Ny);
        if (j < 0) return;
        for (long i = 0; i < Nx; ++i) push_unit(L, j * Nx + i, 1.0 / fabs(tx));
    } else if (tx == 0.0) {
        /* Remark cases_2D (phi = pi/2): the same with the roles of i and j exchanged */
        long i = pick_x(px, Nx);
        if (i < 0) return;
        for (long j = 0; j < Ny; ++j) push_unit(L, j * Nx + i, 1.0 / fabs(ty));
    } else {
        case1_plane(Nx, px, tx, Ny, py, ty, 0, 1, Nx, L);
    }
}

/* 3D: ray point and direction in the scaled frame (R4). */
static void units_3d(const orc_geom *g, double px, double py, double pz, double tx, double ty,
                     double tz, orc_list *L)
{
    const long Nx = g->nx, Ny = g->ny, Nz = g->nz;
    const int zx = (tx == 0.0), zy = (ty == 0.0), zz = (tz == 0.0);
    const int nzero = zx + zy + zz;
    if (nzero == 3) return;
    if (nzero == 2) {
        /* Case 3 (ray along x), its Remark (along y), Case 4 (along z) */
        if (!zx) {
            long j = pick_y(py, Ny), k = pick_y(pz, Nz);
            if (j < 0 || k < 0) return;
            for (long i = 0; i < Nx; ++i) push_unit(L, (k * Ny + j) * Nx + i, 1.0 / fabs(tx));
        } else if (!zy) {
            long i = pick_x(px, Nx), k = pick_y(pz, Nz);
            if (i < 0 || k < 0) return;
            for (long j = 0; j < Ny; ++j) push_unit(L, (k * Ny + j) * Nx + i, 1.0 / fabs(ty));
        } else {
            long i = pick_x(px, Nx), j = pick_y(py, Ny);
            if (i < 0 || j < 0) return;
            for (long k = 0; k < Nz; ++k) push_unit(L, (k * Ny + j) * Nx + i, 1.0 / fabs(tz));
        }
        return;
    }
    if (nzero == 1) {
        if (zy) {
            /* Case 2 (phi1 in {0, pi}): j from the closed range, then the 2D case in (x, z)
             * with C_x, C_z of eq. C_xC_z and the k-range of eq. restriction_k_case2_3D */
            long j = pick_y(py, Ny);
            if (j < 0) return;
            case1_plane(Nx, px, tx, Nz, pz, tz, j * Nx, 1, Nx * Ny, L);
        } else if (zx) {
            /* Remark case2_3D (phi1 in {pi/2, 3pi/2}): i from the closed range, then the 2D
             * case in (y, z), y driving.  y is oriented downwards, so it enters the plane
             * routine through the coordinate -y, whose unit j covers [j - N/2, j - N/2 + 1]. */
            long i = pick_x(px, Nx);
            if (i < 0) return;
            case1_plane(Ny, -py, -ty, Nz, pz, tz, i, Nx, Nx * Ny, L);
        } else {
            /* R5: horizontal oblique ray, k from the closed range, 2D case in (x, y) */
            long k = pick_y(pz, Nz);
            if (k < 0) return;
            case1_plane(Nx, px, tx, Ny, py, ty, k * Nx * Ny, 1, Nx, L);
        }
        return;
    }
    case1_space(g, px, py, pz, tx, ty, tz, L);
}

/* ---------------------------------------------------------------------------------------
 * Ray parameters from the scan (step 1) and the symmetries (step 2)
 * ------------------------------------------------------------------------------------- */

static double det_u(const orc_geom *g, long c) { return (c - 0.5 * (g->n_cols - 1)) * g->du + g->u0; }
static double det_v(const orc_geom *g, long r) { return (r - 0.5 * (g->n_rows - 1)) * g->dv + g->v0; }

/* 2D: (s, phi) of ray (view v, column c) */
static void params_2d(const orc_geom *g, long v, long c, double *s, double *phi)
{
    if (g->kind == K_RAYS2D) {
        /* a ray given by its own parameters (Section 4.3: any ray set whose parameters are
         * known) */
        *s = g->angles[2 * v];
        *phi = g->angles[2 * v + 1];
        return;
    }
    const double u = det_u(g, c), a = g->angles[v], D = g->sod;
    if (g->kind == K_PAR2D) {
        *s = u;
        *phi = a;
    } else if (g->kind == K_FAN2D) {
        /* eq. 2Dparalleltofan_2, t on the line through the origin (R6) */
        const double t = u * g->sod / g->sdd;
        *s = D * t / sqrt(D * D + t * t);
        *phi = atan(t / D) + a - M_PI / 2.0;
    } else {
        /* eq. 2Dparalleltofan, u is the angle gamma */
        *s = D * sin(u);
        *phi = u + a - M_PI / 2.0;
    }
}

/* 3D: (s1, s2, phi1, phi2) of ray (view v, row r, column c) */
static void params_3d(const orc_geom *g, long v, long r, long c, double *s1, double *s2,
                      double *phi1, double *phi2)
{
    if (g->kind == K_RAYS3D) {
        *s1 = g->angles[4 * v];
        *s2 = g->angles[4 * v + 1];
        *phi1 = g->angles[4 * v + 2];
        *phi2 = g->angles[4 * v + 3];
        return;
    }
    const double u = det_u(g, c), w = det_v(g, r), D = g->sod;
    const int helical = (g->kind == K_HELIX || g->kind == K_HELIX_ARC);
    const double H = helical ? g->src_z[v] : 0.0;
    if (g->kind == K_PAR3D) {
        *phi1 = g->angles[2 * v];
        *phi2 = g->angles[2 * v + 1];
        *s1 = u;
        *s2 = w;
    } else if (g->kind == K_CONE || g->kind == K_HELIX) {
        /* eq. equispaced_cone_beam (+ eq. Helical_cone_beam_equispaced), R6 */
        const double t = u * g->sod / g->sdd, h = w * g->sod / g->sdd;
        const double alpha = atan(t / D);
        const double beta = atan(h / sqrt(D * D + t * t));
        *phi1 = g->angles[v] + alpha;
        *phi2 = beta;
        *s1 = D * sin(alpha);
        *s2 = h * cos(alpha) * cos(alpha) * cos(beta) + H * cos(beta);
    } else {
        /* eq. equiangular_cone_beam (+ eq. Helical_cone_beam_equiangular): u, w are the angles */
        const double alpha = u, beta = w;
        *phi1 = g->angles[v] + alpha;
        *phi2 = beta;
        *s1 = D * sin(alpha);
        *s2 = D * cos(alpha) * sin(beta) + H * cos(beta);
    }
}

/* Section 2.2.1: (s, phi + 2n pi) == (s, phi), (s, phi + pi) == (-s, phi) -> phi in [0, pi) */
static void canon_2d(double *s, double *phi)
{
    double p = fmod(*phi, 2.0 * M_PI);
    if (p < 0) p += 2.0 * M_PI;
    if (p >= M_PI) {
        p -= M_PI;
        *s = -*s;
    }
    *phi = p;
}

/* Section 3.2.1: (s1, s2, phi1, phi2 + pi) == (s1, -s2, phi1, phi2) and
 * (-s1, s2, phi1 + pi, -phi2) == (s1, s2, phi1, phi2) -> [0, 2pi) x [0, pi/2] */
static void canon_3d(double *s1, double *s2, double *phi1, double *phi2)
{
    double p2 = fmod(*phi2, 2.0 * M_PI);
    if (p2 > M_PI) p2 -= 2.0 * M_PI;
    if (p2 <= -M_PI) p2 += 2.0 * M_PI;
    if (p2 > M_PI / 2.0) {
        p2 -= M_PI;
        *s2 = -*s2;
    } else if (p2 < -M_PI / 2.0) {
        p2 += M_PI;
        *s2 = -*s2;
    }
    double p1 = *phi1;
    if (p2 < 0) {
        *s1 = -*s1;
        p1 += M_PI;
        p2 = -p2;
    }
    p1 = fmod(p1, 2.0 * M_PI);
    if (p1 < 0) p1 += 2.0 * M_PI;
    *phi1 = p1;
    *phi2 = p2;
}

/* cos/sin of an angle with R7 applied */
static void cos_sin(double a, double *c, double *s)
{
    *c = cos(a);
    *s = sin(a);
    if (fabs(*c) < 1e-12) {
        *c = 0.0;
        *s = (*s > 0) ? 1.0 : -1.0;
    } else if (fabs(*s) < 1e-12) {
        *s = 0.0;
        *c = (*c > 0) ? 1.0 : -1.0;
    }
}

/* Units crossed by ray r with positive length; the list is sorted by 1D index. */
static int cmp_pair(const void *a, const void *b)
{
    const long ia = *(const long *)a, ib = *(const long *)b;
    return (ia > ib) - (ia < ib);
}

static void sort_units(orc_list *L)
{
    if (L->n < 2) return;
    struct pr { long i; double l; } *tmp = malloc(sizeof(*tmp) * (size_t)L->n);
    for (int u = 0; u < L->n; ++u) { tmp[u].i = L->idx[u]; tmp[u].l = L->len[u]; }
    qsort(tmp, (size_t)L->n, sizeof(*tmp), cmp_pair);
    for (int u = 0; u < L->n; ++u) { L->idx[u] = tmp[u].i; L->len[u] = tmp[u].l; }
    free(tmp);
}

static void ray_units(const orc_geom *g, long r, orc_list *L)
{
    L->n = 0;
    L->overflow = 0;
    L->n_trace = 0;
    const long nc = g->n_cols, nr = g->n_rows;
    const long c = r % nc, row = (r / nc) % nr, v = r / (nc * nr);
    if (!is3d(g)) {
        double s, phi;
        params_2d(g, v, c, &s, &phi);
        canon_2d(&s, &phi);
        double cp, sp;
        cos_sin(phi, &cp, &sp);
        /* eq. direction_normal: theta = (cos, sin), point s * theta_perp = s(-sin, cos) */
        const double px = (-s * sp - g->cx) / g->dx, py = (s * cp - g->cy) / g->dy;
        units_2d(g, px, py, cp / g->dx, sp / g->dy, L);
    } else {
        double s1, s2, phi1, phi2;
        params_3d(g, v, row, c, &s1, &s2, &phi1, &phi2);
        canon_3d(&s1, &s2, &phi1, &phi2);
        double c1, sn1, c2, sn2;
        cos_sin(phi1, &c1, &sn1);
        cos_sin(phi2, &c2, &sn2);
        /* eq. 3Dparallel_direction, eq. theta_1, eq. theta_2 */
        const double th[3] = {c2 * c1, c2 * sn1, sn2};
        const double t1[3] = {-sn1, c1, 0.0};
        const double t2[3] = {-sn2 * c1, -sn2 * sn1, c2};
        const double p[3] = {s1 * t1[0] + s2 * t2[0], s1 * t1[1] + s2 * t2[1], s1 * t1[2] + s2 * t2[2]};
        units_3d(g, (p[0] - g->cx) / g->dx, (p[1] - g->cy) / g->dy, (p[2] - g->cz) / g->dz,
                 th[0] / g->dx, th[1] / g->dy, th[2] / g->dz, L);
    }
    sort_units(L);
}

static int list_cap(const orc_geom *g) { return 4 * (g->nx + g->ny + g->nz) + 16; }

static void list_init(orc_list *L, int cap)
{
    memset(L, 0, sizeof(*L));
    L->idx = malloc(sizeof(long) * (size_t)cap);
    L->len = malloc(sizeof(double) * (size_t)cap);
    L->cap = cap;
}

static void list_free(orc_list *L)
{
    free(L->idx);
    free(L->len);
}

/* ---------------------------------------------------------------------------------------
 * Exported entry points (ctypes)
 * ------------------------------------------------------------------------------------- */

/* Canonical ray parameters: 2D writes (s, phi), 3D writes (s1, s2, phi1, phi2). */
void orc_ray_params(const orc_geom *g, long r, double *out)
{
    const long nc = g->n_cols, nr = g->n_rows;
    const long c = r % nc, row = (r / nc) % nr, v = r / (nc * nr);
    if (!is3d(g)) {
        params_2d(g, v, c, &out[0], &out[1]);
        canon_2d(&out[0], &out[1]);
    } else {
        params_3d(g, v, row, c, &out[0], &out[1], &out[2], &out[3]);
        canon_3d(&out[0], &out[1], &out[2], &out[3]);
    }
}

/* Sparse row of the projection matrix for ray r (Algorithm 1/2 "Output"): indices sorted
 * ascending.  Returns the number of units (-1 if cap was too small). */
int orc_ray_units(const orc_geom *g, long r, long *idx, double *len, int cap, double *trace,
                  int cap_trace, int *n_trace)
{
    orc_list L;
    list_init(&L, list_cap(g));
    L.trace = trace;
    L.cap_trace = cap_trace;
    ray_units(g, r, &L);
    int n = L.n;
    if (L.overflow || n > cap) n = -1;
    else {
        memcpy(idx, L.idx, sizeof(long) * (size_t)L.n);
        memcpy(len, L.len, sizeof(double) * (size_t)L.n);
    }
    if (n_trace) *n_trace = L.n_trace;
    list_free(&L);
    return n;
}

/* Forward projection, eq. Xray_transform_image: sino[b][q] = sum_I img[b][I] * l_I(ray)
 * summed in ascending I.  rays: list of n_rays ray ids, or NULL for every ray (then
 * n_rays must equal the scan's ray count).  img: [batch][units], sino: [batch][n_rays]. */
int orc_forward(const orc_geom *g, const double *img, double *sino, const long *rays,
                long n_rays, int batch, int nthreads)
{
    const long n_units = (long)g->nx * g->ny * g->nz;
    int bad = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1) reduction(| : bad)
    {
        orc_list L;
        list_init(&L, list_cap(g));
#pragma omp for schedule(dynamic, 16)
        for (long q = 0; q < n_rays; ++q) {
            const long r = rays ? rays[q] : q;
            ray_units(g, r, &L);
            if (L.overflow) bad = 1;
            for (int b = 0; b < batch; ++b) {
                const double *f = img + (size_t)b * n_units;
                double acc = 0.0;
                for (int u = 0; u < L.n; ++u) acc += f[L.idx[u]] * L.len[u];
                sino[(size_t)b * n_rays + q] = acc;
            }
        }
        list_free(&L);
    }
    return bad ? -1 : 0;
}

/* Adjoint (backprojection), the transpose of the forward operator (Section 1):
 * img[b][I] = sum over rays of l_I(ray) * sino[b][q].  img is overwritten. */
int orc_adjoint(const orc_geom *g, const double *sino, double *img, const long *rays, long n_rays,
                int batch, int nthreads)
{
    const long n_units = (long)g->nx * g->ny * g->nz;
    memset(img, 0, sizeof(double) * (size_t)n_units * (size_t)batch);
    int bad = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1) reduction(| : bad)
    {
        orc_list L;
        list_init(&L, list_cap(g));
#pragma omp for schedule(dynamic, 16)
        for (long q = 0; q < n_rays; ++q) {
            const long r = rays ? rays[q] : q;
            ray_units(g, r, &L);
            if (L.overflow) bad = 1;
            for (int b = 0; b < batch; ++b) {
                const double gv = sino[(size_t)b * n_rays + q];
                if (gv == 0.0) continue;
                double *f = img + (size_t)b * n_units;
                for (int u = 0; u < L.n; ++u) {
#pragma omp atomic update
                    f[L.idx[u]] += L.len[u] * gv;
                }
            }
        }
        list_free(&L);
    }
    return bad ? -1 : 0;
}

/* ---------------------------------------------------------------------------------------
 * Attenuated transform: the generalized Radon transform of eq. generalizedRadontransform
 * with the exponential attenuation weight of the SPECT case,
 *   Phi(theta, x, t) = exp(-int_t^inf mu(x + s theta) ds),
 * mu a unit image (R15: attenuation is integrated along +theta, the direction of the ray's
 * own parameters before the symmetries are applied).  With f and mu constant on each unit,
 * for the units k of a ray in the order of increasing t, lengths l_k and
 * A_k = sum_{m > k} mu_m l_m:
 *   g = sum_k f_k exp(-A_k) int_0^{l_k} exp(-mu_k (l_k - t)) dt
 *     = sum_k f_k exp(-A_k) (1 - exp(-mu_k l_k)) / mu_k      (l_k when mu_k = 0).
 * ------------------------------------------------------------------------------------- */

/* int_0^l exp(-mu (l - t)) dt */
static double expo_len(double mu, double l)
{
    const double a = mu * l;
    return a != 0.0 ? -expm1(-a) / mu : l;
}

/* Direction theta of ray r from its own parameters (eq. direction_normal / 3Dparallel_direction). */
static void ray_direction(const orc_geom *g, long r, double th[3])
{
    const long nc = g->n_cols, nr = g->n_rows;
    const long c = r % nc, row = (r / nc) % nr, v = r / (nc * nr);
    if (!is3d(g)) {
        double s, phi;
        params_2d(g, v, c, &s, &phi);
        th[0] = cos(phi);
        th[1] = sin(phi);
        th[2] = 0.0;
    } else {
        double s1, s2, phi1, phi2;
        params_3d(g, v, row, c, &s1, &s2, &phi1, &phi2);
        th[0] = cos(phi2) * cos(phi1);
        th[1] = cos(phi2) * sin(phi1);
        th[2] = sin(phi2);
    }
}

typedef struct {
    double key;
    long i;
    double l;
} orc_along;

static int cmp_along(const void *a, const void *b)
{
    const double x = ((const orc_along *)a)->key, y = ((const orc_along *)b)->key;
    return (x > y) - (x < y);
}

/* Weights w_k = exp(-A_k) * expo_len(mu_k, l_k) of the units of L (any order), in place of
 * the lengths.  The crossed units are ordered along theta by their centres' projections:
 * consecutive units of a line share a face (or an edge or corner at a touch), and the centre
 * moves by d_a along each axis the line advances on, in the direction of theta. */
static void attenuate(const orc_geom *g, long r, const double *mu, orc_list *L, orc_along *tmp)
{
    double th[3];
    ray_direction(g, r, th);
    const long nxy = (long)g->nx * g->ny;
    for (int u = 0; u < L->n; ++u) {
        const long I = L->idx[u], k = I / nxy, j = (I % nxy) / g->nx, i = I % g->nx;
        const double x = g->cx + (i + 0.5 - 0.5 * g->nx) * g->dx;
        const double y = g->cy + (0.5 * g->ny - j - 0.5) * g->dy;
        const double z = g->cz + (0.5 * g->nz - k - 0.5) * g->dz;
        tmp[u].key = x * th[0] + y * th[1] + z * th[2];
        tmp[u].i = I;
        tmp[u].l = L->len[u];
    }
    qsort(tmp, (size_t)L->n, sizeof(*tmp), cmp_along);
    double A = 0.0; /* attenuation after the current unit: walk from the far end */
    for (int u = L->n - 1; u >= 0; --u) {
        const double m = mu[tmp[u].i];
        L->idx[u] = tmp[u].i;
        L->len[u] = exp(-A) * expo_len(m, tmp[u].l);
        A += m * tmp[u].l;
    }
}

/* Attenuated forward: sino[b][q] = sum_k img[b][I_k] w_k(ray), mu: [units]. */
int orc_forward_attenuated(const orc_geom *g, const double *mu, const double *img, double *sino, const long *rays,
                           long n_rays, int batch, int nthreads)
{
    const long n_units = (long)g->nx * g->ny * g->nz;
    int bad = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1) reduction(| : bad)
    {
        orc_list L;
        list_init(&L, list_cap(g));
        orc_along *tmp = malloc(sizeof(orc_along) * (size_t)L.cap);
#pragma omp for schedule(dynamic, 16)
        for (long q = 0; q < n_rays; ++q) {
            const long r = rays ? rays[q] : q;
            ray_units(g, r, &L);
            if (L.overflow) bad = 1;
            attenuate(g, r, mu, &L, tmp);
            for (int b = 0; b < batch; ++b) {
                const double *f = img + (size_t)b * n_units;
                double acc = 0.0;
                for (int u = 0; u < L.n; ++u) acc += f[L.idx[u]] * L.len[u];
                sino[(size_t)b * n_rays + q] = acc;
            }
        }
        free(tmp);
        list_free(&L);
    }
    return bad ? -1 : 0;
}

/* Its adjoint: img[b][I] = sum over rays of w_I(ray) * sino[b][q].  img is overwritten. */
int orc_adjoint_attenuated(const orc_geom *g, const double *mu, const double *sino, double *img, const long *rays,
                           long n_rays, int batch, int nthreads)
{
    const long n_units = (long)g->nx * g->ny * g->nz;
    memset(img, 0, sizeof(double) * (size_t)n_units * (size_t)batch);
    int bad = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1) reduction(| : bad)
    {
        orc_list L;
        list_init(&L, list_cap(g));
        orc_along *tmp = malloc(sizeof(orc_along) * (size_t)L.cap);
#pragma omp for schedule(dynamic, 16)
        for (long q = 0; q < n_rays; ++q) {
            const long r = rays ? rays[q] : q;
            ray_units(g, r, &L);
            if (L.overflow) bad = 1;
            attenuate(g, r, mu, &L, tmp);
            for (int b = 0; b < batch; ++b) {
                const double gv = sino[(size_t)b * n_rays + q];
                if (gv == 0.0) continue;
                double *f = img + (size_t)b * n_units;
                for (int u = 0; u < L.n; ++u) {
#pragma omp atomic update
                    f[L.idx[u]] += L.len[u] * gv;
                }
            }
        }
        free(tmp);
        list_free(&L);
    }
    return bad ? -1 : 0;
}

/* Number of OpenMP threads the oracle would use by default (1 without OpenMP). */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
