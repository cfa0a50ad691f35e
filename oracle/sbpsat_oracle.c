/*
 * FP64 CPU oracle for the three-dimensional SBP-SAT FDTD method
 * (arXiv 2206.00638).  TEST INFRASTRUCTURE ONLY: it exists to check the
 * CUDA path.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load it; the product path never does.
 * It shares no source, header, table or helper with the CUDA library.
 *
 * What it computes, in the paper's order and notation:
 *   - 1D staggered grids x+ (n+1 nodes) and x- (n+2 nodes)         Sec. II-A
 *   - 3D field grids per component                                  Table I
 *   - SBP operators D+ = P+^-1 Q+, D- = P-^-1 Q-, rows and weights   Appendix
 *   - semi-discrete Maxwell equations, Kronecker-extended operators  Eqs. (7)-(12)
 *   - PEC SAT on the H equations, sign per face                      Eqs. (13)-(15), (18)
 *   - PMC SAT on the E equations                                     Eqs. (19)-(21), (23)
 *   - block interface SAT: the periodic SAT of Eqs. (EPBC1-6) with
 *     zero phase and the +-1/2 coefficients of Eq. (EPBCP), coupling one
 *     block face to another block's face (conforming)
 *   - periodic SAT with a phase shift (Eqs. (EPBC1-6)): a complex field is
 *     a pair of blocks (real part, imaginary part); the penalty at a high
 *     face compares with e^{-j alpha} times the low-face field, at a low
 *     face with e^{+j alpha} times the high-face field, so each face's
 *     partner value is w_a (partner) + w_b (second partner) with
 *     (w_a, w_b) = (cos alpha, +-sin alpha)
 *   - absorbing SAT: first-order characteristic (Silver-Mueller) penalty,
 *     not in the paper (it uses CPML); energy-dissipative by construction
 *   - leapfrog in time, U^n = [E^n, H^{n-1/2}]                       Sec. IV, Sec. V
 *   - discrete energy with the P''' norms                            Eq. (16)
 *
 * Readings where the paper is silent or garbled:
 *   - D+/D- carry 1/h; eps and mu multiply the whole right-hand side,
 *     SAT terms included (Appendix prints 1/eps, 1/mu without h).
 *   - SAT sign of a pair (E_t, H_t) on a face is phi = -s * side, where s
 *     is the sign the pair carries in Eqs. (7)-(12) and side = -1 / +1 for
 *     a low / high face.  This reproduces every entry of Eqs. (18), (23).
 *   - node permittivity/permeability = arithmetic mean over the cells
 *     whose closed box contains the node.
 *   - absorbing self terms are time-averaged over the two levels of the
 *     update (pointwise semi-implicit), keeping the scheme explicit.
 *   - energy monitor: the leapfrog-consistent form
 *       W^n = 1/2 [ sum_E eps P''' (E^n)^2 + sum_H mu P''' H^{n-1/2} H^{n+1/2} ]
 *     which reduces to Eq. (16) as dt -> 0 and is exactly conserved by
 *     leapfrog for energy-neutral SATs.
 *
 * Layout: each component is stored in its natural extents (n+1 along a
 * plus-grid axis, n+2 along a minus-grid axis), x fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OB_C0 299792458.0
#define OB_EPS0 8.8541878128e-12
#define OB_MU0 1.25663706212e-6
#define OB_PI 3.14159265358979323846

enum { OB_PEC = 0, OB_PMC = 1, OB_ABS = 2, OB_IFACE = 3 };
enum { EX = 0, EY, EZ, HX, HY, HZ };
enum { WF_GAUSS = 0, WF_GAUSS_DERIV = 1, WF_MOD_GAUSS = 2 };

/* Table I: 1 if component c lives on the plus grid along axis a. */
static const int ON_PLUS[6][3] = {
    {0, 1, 1}, /* Ex: x-, y+, z+ */
    {1, 0, 1}, /* Ey: x+, y-, z+ */
    {1, 1, 0}, /* Ez: x+, y+, z- */
    {1, 0, 0}, /* Hx: x+, y-, z- */
    {0, 1, 0}, /* Hy: x-, y+, z- */
    {0, 0, 1}, /* Hz: x-, y-, z+ */
};

/* Eqs. (7)-(12): dC/dt = sgn0 * D^{ax0} C0 + sgn1 * D^{ax1} C1 */
typedef struct { int sgn, comp, axis; } ob_term;
static const ob_term CURL[6][2] = {
    {{+1, HZ, 1}, {-1, HY, 2}}, /* (7)  dEx = Dy Hz - Dz Hy */
    {{+1, HX, 2}, {-1, HZ, 0}}, /* (8)  dEy = Dz Hx - Dx Hz */
    {{+1, HY, 0}, {-1, HX, 1}}, /* (9)  dEz = Dx Hy - Dy Hx */
    {{+1, EY, 2}, {-1, EZ, 1}}, /* (10) dHx = Dz Ey - Dy Ez */
    {{+1, EZ, 0}, {-1, EX, 2}}, /* (11) dHy = Dx Ez - Dz Ex */
    {{+1, EX, 1}, {-1, EY, 0}}, /* (12) dHz = Dy Ex - Dx Ey */
};

/* ---------------------------------------------------------------- */
/* 1D operators of the Appendix (unit spacing).                      */
/* ---------------------------------------------------------------- */
typedef struct { int col0, ncol; double c[3]; } ob_row;

/* Row r of D+ (size (n+1) x (n+2)): derivative on x+ from values on x-. */
static ob_row dplus_row(int n, int r)
{
    ob_row R;
    if (r == 0) {
        R.col0 = 0; R.ncol = 3; R.c[0] = -1.0; R.c[1] = 0.5; R.c[2] = 0.5;
    } else if (r == 1) {
        R.col0 = 0; R.ncol = 3; R.c[0] = -0.5; R.c[1] = -0.25; R.c[2] = 0.75;
    } else if (r == n - 1) {
        R.col0 = n - 1; R.ncol = 3; R.c[0] = -0.75; R.c[1] = 0.25; R.c[2] = 0.5;
    } else if (r == n) {
        R.col0 = n - 1; R.ncol = 3; R.c[0] = -0.5; R.c[1] = -0.5; R.c[2] = 1.0;
    } else {
        R.col0 = r; R.ncol = 2; R.c[0] = -1.0; R.c[1] = 1.0; R.c[2] = 0.0;
    }
    return R;
}

/* Row r of D- (size (n+2) x (n+1)): derivative on x- from values on x+. */
static ob_row dminus_row(int n, int r)
{
    ob_row R;
    R.c[2] = 0.0;
    if (r == 0 || r == 1) {
        R.col0 = 0; R.ncol = 2; R.c[0] = -1.0; R.c[1] = 1.0;
    } else if (r == 2) {
        R.col0 = 0; R.ncol = 3; R.c[0] = -1.0 / 5.0; R.c[1] = -3.0 / 5.0; R.c[2] = 4.0 / 5.0;
    } else if (r == n - 1) {
        R.col0 = n - 2; R.ncol = 3; R.c[0] = -4.0 / 5.0; R.c[1] = 3.0 / 5.0; R.c[2] = 1.0 / 5.0;
    } else if (r == n || r == n + 1) {
        R.col0 = n - 1; R.ncol = 2; R.c[0] = -1.0; R.c[1] = 1.0;
    } else {
        R.col0 = r - 1; R.ncol = 2; R.c[0] = -1.0; R.c[1] = 1.0;
    }
    return R;
}

/* Diagonal norms (unit spacing): P+ = diag(1/2,1,...,1,1/2),
 * P- = diag(1/2,1/4,5/4,1,...,1,5/4,1/4,1/2). */
static double pplus(int n, int r) { return (r == 0 || r == n) ? 0.5 : 1.0; }
static double pminus(int n, int r)
{
    if (r == 0 || r == n + 1) return 0.5;
    if (r == 1 || r == n) return 0.25;
    if (r == 2 || r == n - 1) return 1.25;
    return 1.0;
}

void ob_dplus(int n, double *out)
{
    memset(out, 0, sizeof(double) * (size_t)(n + 1) * (n + 2));
    for (int r = 0; r <= n; r++) {
        ob_row R = dplus_row(n, r);
        for (int q = 0; q < R.ncol; q++) out[(size_t)r * (n + 2) + R.col0 + q] = R.c[q];
    }
}
void ob_dminus(int n, double *out)
{
    memset(out, 0, sizeof(double) * (size_t)(n + 2) * (n + 1));
    for (int r = 0; r <= n + 1; r++) {
        ob_row R = dminus_row(n, r);
        for (int q = 0; q < R.ncol; q++) out[(size_t)r * (n + 1) + R.col0 + q] = R.c[q];
    }
}
void ob_pplus(int n, double *out) { for (int r = 0; r <= n; r++) out[r] = pplus(n, r); }
void ob_pminus(int n, double *out) { for (int r = 0; r <= n + 1; r++) out[r] = pminus(n, r); }

/* ---------------------------------------------------------------- */
/* Blocks                                                            */
/* ---------------------------------------------------------------- */
typedef struct { int comp, idx[3], wf; double amp, tw, t0, f; } ob_source;
typedef struct { int comp, idx[3]; } ob_probe;

typedef struct ob_block {
    int n[3];
    double h[3];
    double dt;
    int face[6];                 /* x-, x+, y-, y+, z-, z+ */
    struct ob_block *nbr[6];
    int nbr_face[6];
    struct ob_block *nbr2[6];    /* second partner of a phase-shifted periodic face (NULL: none) */
    double nbr_w[6][2];          /* partner value = w[0] nbr + w[1] nbr2 */
    double *cell_eps, *cell_mu;  /* relative, n0*n1*n2, x fastest */
    double *F[6];                /* fields, natural extents */
    double *epsn[6], *mun[6];    /* relative node eps, mu on each component grid */
    double *rhs[6];
    double *tmp[3];              /* trial H^{n+1/2} for the energy */
    ob_source *src; int nsrc;
    ob_probe *prb; int nprb;
    double *prb_buf; long prb_cap;
    long step;
} ob_block;

static int ext(const ob_block *b, int c, int a) { return b->n[a] + (ON_PLUS[c][a] ? 1 : 2); }
static size_t count(const ob_block *b, int c) { return (size_t)ext(b, c, 0) * ext(b, c, 1) * ext(b, c, 2); }
static size_t at(const ob_block *b, int c, int i, int j, int k)
{
    return ((size_t)k * ext(b, c, 1) + j) * ext(b, c, 0) + i;
}

/* 1D weight of node r of component c along axis a, including h (Appendix). */
static double w1(const ob_block *b, int c, int a, int r)
{
    return b->h[a] * (ON_PLUS[c][a] ? pplus(b->n[a], r) : pminus(b->n[a], r));
}

/* Node position along an axis in units of h/2: plus node p at p*h,
 * minus node 0 at 0, m in 1..n at (m-1/2)h, n+1 at n*h. */
static int half_pos(int plus, int n, int r)
{
    if (plus) return 2 * r;
    if (r == 0) return 0;
    if (r == n + 1) return 2 * n;
    return 2 * r - 1;
}

/* Mean of a cell array over the cells whose closed box contains the node. */
static double node_mean(const ob_block *b, const double *cells, int c, int i, int j, int k)
{
    if (!cells) return 1.0;
    int idx[3] = {i, j, k};
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        int p = half_pos(ON_PLUS[c][a], b->n[a], idx[a]);
        lo[a] = b->n[a]; hi[a] = -1;
        for (int cell = 0; cell < b->n[a]; cell++) {
            if (2 * cell <= p && p <= 2 * cell + 2) {
                if (cell < lo[a]) lo[a] = cell;
                if (cell > hi[a]) hi[a] = cell;
            }
        }
    }
    double s = 0.0; int cnt = 0;
    for (int z = lo[2]; z <= hi[2]; z++)
        for (int y = lo[1]; y <= hi[1]; y++)
            for (int x = lo[0]; x <= hi[0]; x++) {
                s += cells[((size_t)z * b->n[1] + y) * b->n[0] + x];
                cnt++;
            }
    return s / cnt;
}

ob_block *ob_create(int nx, int ny, int nz, double dx, double dy, double dz, double dt,
                    const int *faces, const double *eps_cells, const double *mu_cells)
{
    if (nx < 4 || ny < 4 || nz < 4) return NULL;
    ob_block *b = (ob_block *)calloc(1, sizeof(ob_block));
    b->n[0] = nx; b->n[1] = ny; b->n[2] = nz;
    b->h[0] = dx; b->h[1] = dy; b->h[2] = dz;
    b->dt = dt;
    for (int f = 0; f < 6; f++) {
        b->face[f] = faces[f]; b->nbr[f] = NULL; b->nbr_face[f] = -1;
        b->nbr2[f] = NULL; b->nbr_w[f][0] = 1.0; b->nbr_w[f][1] = 0.0;
    }
    size_t ncell = (size_t)nx * ny * nz;
    if (eps_cells) { b->cell_eps = (double *)malloc(ncell * sizeof(double)); memcpy(b->cell_eps, eps_cells, ncell * sizeof(double)); }
    if (mu_cells) { b->cell_mu = (double *)malloc(ncell * sizeof(double)); memcpy(b->cell_mu, mu_cells, ncell * sizeof(double)); }
    for (int c = 0; c < 6; c++) {
        size_t m = count(b, c);
        b->F[c] = (double *)calloc(m, sizeof(double));
        b->rhs[c] = (double *)calloc(m, sizeof(double));
        b->epsn[c] = (double *)malloc(m * sizeof(double));
        b->mun[c] = (double *)malloc(m * sizeof(double));
        int e0 = ext(b, c, 0), e1 = ext(b, c, 1), e2 = ext(b, c, 2);
#pragma omp parallel for schedule(static)
        for (int k = 0; k < e2; k++)
            for (int j = 0; j < e1; j++)
                for (int i = 0; i < e0; i++) {
                    b->epsn[c][at(b, c, i, j, k)] = node_mean(b, b->cell_eps, c, i, j, k);
                    b->mun[c][at(b, c, i, j, k)] = node_mean(b, b->cell_mu, c, i, j, k);
                }
    }
    for (int c = 0; c < 3; c++) b->tmp[c] = (double *)calloc(count(b, HX + c), sizeof(double));
    return b;
}

void ob_destroy(ob_block *b)
{
    if (!b) return;
    for (int c = 0; c < 6; c++) { free(b->F[c]); free(b->rhs[c]); free(b->epsn[c]); free(b->mun[c]); }
    for (int c = 0; c < 3; c++) free(b->tmp[c]);
    free(b->cell_eps); free(b->cell_mu); free(b->src); free(b->prb); free(b->prb_buf);
    free(b);
}

long ob_count(const ob_block *b, int c) { return (long)count(b, c); }
void ob_set_field(ob_block *b, int c, const double *src) { memcpy(b->F[c], src, count(b, c) * sizeof(double)); }
void ob_get_field(const ob_block *b, int c, double *dst) { memcpy(dst, b->F[c], count(b, c) * sizeof(double)); }
void ob_get_rhs(const ob_block *b, int c, double *dst) { memcpy(dst, b->rhs[c], count(b, c) * sizeof(double)); }
void ob_get_node_eps(const ob_block *b, int c, double *dst) { memcpy(dst, b->epsn[c], count(b, c) * sizeof(double)); }
long ob_get_step(const ob_block *b) { return b->step; }
void ob_set_step(ob_block *b, long s) { b->step = s; }

/* Conforming interface between face fa of a and face fb of b: the two
 * faces must be normal to the same axis, have opposite sides, and share
 * the transverse node sets (cell counts and spacings). */
int ob_connect(ob_block *a, int fa, ob_block *b, int fb)
{
    int ax = fa / 2, bx = fb / 2;
    if (ax != bx || (fa % 2) == (fb % 2)) return -1;
    for (int t = 0; t < 3; t++) {
        if (t == ax) continue;
        if (a->n[t] != b->n[t] || a->h[t] != b->h[t]) return -2;
    }
    a->face[fa] = OB_IFACE; b->face[fb] = OB_IFACE;
    a->nbr[fa] = b; a->nbr_face[fa] = fb;
    b->nbr[fb] = a; b->nbr_face[fb] = fa;
    a->nbr2[fa] = NULL; a->nbr_w[fa][0] = 1.0; a->nbr_w[fa][1] = 0.0;
    b->nbr2[fb] = NULL; b->nbr_w[fb][0] = 1.0; b->nbr_w[fb][1] = 0.0;
    return 0;
}

/* Periodic faces along `axis` with phase shift alpha (Eqs. (EPBC1-6)) for the
 * complex field re + j im held by two blocks of equal shape.  The field one
 * period above equals e^{-j alpha} times the field here, so
 *   high face:  C_high - e^{-j alpha} C_low,   low face:  C_low - e^{+j alpha} C_high
 * (C the partner component).  With e^{-+j alpha}(a + j b) split into real and
 * imaginary parts, the partner value seen by
 *   re, high: cos a * re_low  + sin a * im_low      re, low: cos a * re_high - sin a * im_high
 *   im, high: cos a * im_low  - sin a * re_low      im, low: cos a * im_high + sin a * re_high */
int ob_connect_phase(ob_block *re, ob_block *im, int axis, double alpha)
{
    if (axis < 0 || axis > 2 || re == im) return -1;
    for (int t = 0; t < 3; t++)
        if (re->n[t] != im->n[t] || re->h[t] != im->h[t]) return -2;
    const double c = cos(alpha), s = sin(alpha);
    const int lo = 2 * axis, hi = 2 * axis + 1;
    ob_block *own[2] = {re, im}, *other[2] = {im, re};
    const double wb_hi[2] = {+s, -s}, wb_lo[2] = {-s, +s};
    for (int q = 0; q < 2; q++) {
        ob_block *b = own[q];
        b->face[lo] = OB_IFACE; b->face[hi] = OB_IFACE;
        b->nbr[hi] = b; b->nbr_face[hi] = lo; b->nbr2[hi] = other[q];
        b->nbr_w[hi][0] = c; b->nbr_w[hi][1] = wb_hi[q];
        b->nbr[lo] = b; b->nbr_face[lo] = hi; b->nbr2[lo] = other[q];
        b->nbr_w[lo][0] = c; b->nbr_w[lo][1] = wb_lo[q];
    }
    return 0;
}

int ob_add_source(ob_block *b, int comp, int i, int j, int k, int wf, double amp, double tw, double t0, double f)
{
    b->src = (ob_source *)realloc(b->src, sizeof(ob_source) * (b->nsrc + 1));
    ob_source *s = &b->src[b->nsrc];
    s->comp = comp; s->idx[0] = i; s->idx[1] = j; s->idx[2] = k;
    s->wf = wf; s->amp = amp; s->tw = tw; s->t0 = t0; s->f = f;
    return b->nsrc++;
}

int ob_add_probe(ob_block *b, int comp, int i, int j, int k)
{
    b->prb = (ob_probe *)realloc(b->prb, sizeof(ob_probe) * (b->nprb + 1));
    ob_probe *p = &b->prb[b->nprb];
    p->comp = comp; p->idx[0] = i; p->idx[1] = j; p->idx[2] = k;
    return b->nprb++;
}

/* Reserve room for nsteps of probe samples; sample s of probe p is stored at p*cap + s. */
void ob_probe_reserve(ob_block *b, long cap)
{
    free(b->prb_buf);
    b->prb_cap = cap;
    b->prb_buf = (double *)calloc((size_t)(b->nprb > 0 ? b->nprb : 1) * cap, sizeof(double));
}
void ob_get_probes(const ob_block *b, double *dst)
{
    memcpy(dst, b->prb_buf, sizeof(double) * (size_t)b->nprb * b->prb_cap);
}

/* Source waveforms: the Gaussian pulse exp(-4 pi (t-t0)^2 / tw^2) (Sec. VI-B),
 * its time derivative normalised to unit peak, and the modulated Gaussian
 * sin(2 pi f t) exp(-4 pi (t-t0)^2 / tw^2) (Sec. VI-C). */
double ob_waveform(int wf, double t, double tw, double t0, double f)
{
    double x = t - t0;
    double g = exp(-4.0 * OB_PI * x * x / (tw * tw));
    if (wf == WF_GAUSS) return g;
    if (wf == WF_GAUSS_DERIV) return -sqrt(8.0 * OB_PI) * (x / tw) * exp(0.5) * g;
    return sin(2.0 * OB_PI * f * t) * g;
}

/* dt = cfl / (c sqrt(1/dx^2 + 1/dy^2 + 1/dz^2)): the FDTD limit, which the
 * paper states is also the SBP-SAT limit (Sec. VI-A). */
double ob_dt(double cfl, double dx, double dy, double dz, double c)
{
    return cfl / (c * sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz)));
}

/* ---------------------------------------------------------------- */
/* Semi-discrete right-hand side                                      */
/* ---------------------------------------------------------------- */

/* Derivative along axis a of component u at the node idx of the output grid
 * (the complementary grid of u along a), one row of D+ or D- with 1/h. */
static double deriv(const ob_block *b, int u, int a, const int idx[3])
{
    int n = b->n[a];
    ob_row R = ON_PLUS[u][a] ? dminus_row(n, idx[a]) : dplus_row(n, idx[a]);
    int q[3] = {idx[0], idx[1], idx[2]};
    double s = 0.0;
    for (int t = 0; t < R.ncol; t++) {
        q[a] = R.col0 + t;
        s += R.c[t] * b->F[u][at(b, u, q[0], q[1], q[2])];
    }
    return s / b->h[a];
}

/* Tangential partner of component c for a face normal to axis: the field
 * that c's equation differentiates along that axis, and the sign s the pair
 * carries in Eqs. (7)-(12); -1 if c is normal to the face. */
static int partner(int c, int axis, int *s)
{
    for (int t = 0; t < 2; t++) {
        /* the term of c's equation that differentiates along axis */
        if (CURL[c][t].axis == axis) { *s = CURL[c][t].sgn; return CURL[c][t].comp; }
    }
    return -1;
}

/* SAT contributions at a node of component c:
 *   *expl  += explicit penalty (partner values, neighbour values), before the
 *             material factor 1/eps or 1/mu;
 *   *self  += coefficient g of the self term  -g * C  (absorbing faces).
 * Follows sigma (P''')^-1 R^T P'' (.) of Eqs. (13)-(15), chi ... of
 * Eqs. (19)-(21) and the zero-phase form of Eqs. (EPBC1-6). */
static void sat_terms(const ob_block *b, int c, const int idx[3], double eps_r, double mu_r,
                      double *expl, double *self)
{
    int isH = c >= HX;
    for (int f = 0; f < 6; f++) {
        int ax = f / 2, side = (f % 2) ? +1 : -1;
        if (idx[ax] != 0 && idx[ax] != ext(b, c, ax) - 1) continue;   /* not on this face */
        int s; int p = partner(c, ax, &s);
        if (p < 0) continue;                     /* c is normal to this face */
        /* the tangential field on a face sits on the end nodes of its grid */
        int end = (side < 0) ? 0 : ext(b, c, ax) - 1;
        if (idx[ax] != end) continue;
        int type = b->face[f];
        if (isH && type == OB_PMC) continue;
        if (!isH && type == OB_PEC) continue;
        double phi = -(double)s * side;
        /* (P''')^-1 R^T P'': transverse weights cancel against P''', leaving
         * the reciprocal of the end weight along the normal. */
        double wt = 1.0, wf = 1.0;
        for (int a = 0; a < 3; a++) {
            double w = w1(b, c, a, idx[a]);
            wt *= w;
            if (a != ax) wf *= w;
        }
        double ratio = wf / wt;
        int pidx[3] = {idx[0], idx[1], idx[2]};
        pidx[ax] = (side < 0) ? 0 : ext(b, p, ax) - 1;
        double pv = b->F[p][at(b, p, pidx[0], pidx[1], pidx[2])];
        if (type == OB_PEC || type == OB_PMC) {
            *expl += phi * ratio * pv;
        } else if (type == OB_ABS) {
            double eta = sqrt(OB_MU0 * mu_r / (OB_EPS0 * eps_r));
            *expl += phi * ratio * 0.5 * pv;
            *self += ratio * (isH ? 0.5 * eta : 0.5 / eta);
        } else { /* OB_IFACE */
            const ob_block *nb = b->nbr[f];
            int nf = b->nbr_face[f];
            int nside = (nf % 2) ? +1 : -1;
            int q[3] = {idx[0], idx[1], idx[2]};
            q[ax] = (nside < 0) ? 0 : ext(nb, p, ax) - 1;
            const size_t qo = at(nb, p, q[0], q[1], q[2]);
            double nv = b->nbr_w[f][0] * nb->F[p][qo];
            if (b->nbr2[f]) nv += b->nbr_w[f][1] * b->nbr2[f]->F[p][qo];
            *expl += phi * ratio * 0.5 * (pv - nv);
        }
    }
}

/* Right-hand side (explicit part L, self coefficient g) at one node:
 * dC/dt = L - g C  with the material factor applied. */
static void node_rhs(const ob_block *b, int c, const int idx[3], double *L, double *g)
{
    size_t o = at(b, c, idx[0], idx[1], idx[2]);
    double er = b->epsn[c][o], mr = b->mun[c][o];
    double curl = 0.0;
    for (int t = 0; t < 2; t++) curl += CURL[c][t].sgn * deriv(b, CURL[c][t].comp, CURL[c][t].axis, idx);
    double expl = 0.0, self = 0.0;
    sat_terms(b, c, idx, er, mr, &expl, &self);
    double m = (c >= HX) ? OB_MU0 * mr : OB_EPS0 * er;
    *L = (curl + expl) / m;
    *g = self / m;
}

/* dU/dt of the semi-discrete system (no sources) for all blocks. */
void ob_rhs(ob_block **blocks, int nb)
{
    for (int bi = 0; bi < nb; bi++) {
        ob_block *b = blocks[bi];
        for (int c = 0; c < 6; c++) {
            int e0 = ext(b, c, 0), e1 = ext(b, c, 1), e2 = ext(b, c, 2);
#pragma omp parallel for schedule(static)
            for (int k = 0; k < e2; k++)
                for (int j = 0; j < e1; j++)
                    for (int i = 0; i < e0; i++) {
                        int idx[3] = {i, j, k};
                        double L, g;
                        node_rhs(b, c, idx, &L, &g);
                        b->rhs[c][at(b, c, i, j, k)] = L - g * b->F[c][at(b, c, i, j, k)];
                    }
        }
    }
}

/* ---------------------------------------------------------------- */
/* Leapfrog                                                          */
/* ---------------------------------------------------------------- */

/* H^{n+1/2} from E^n and H^{n-1/2} into dst (may alias F[H]). */
static void h_half_step(ob_block *b, double *dst[3])
{
    double dt = b->dt;
    for (int c = HX; c <= HZ; c++) {
        int e0 = ext(b, c, 0), e1 = ext(b, c, 1), e2 = ext(b, c, 2);
#pragma omp parallel for schedule(static)
        for (int k = 0; k < e2; k++)
            for (int j = 0; j < e1; j++)
                for (int i = 0; i < e0; i++) {
                    int idx[3] = {i, j, k};
                    double L, g;
                    node_rhs(b, c, idx, &L, &g);
                    size_t o = at(b, c, i, j, k);
                    double old = b->F[c][o];
                    dst[c - HX][o] = ((1.0 - 0.5 * dt * g) * old + dt * L) / (1.0 + 0.5 * dt * g);
                }
    }
}

static double source_value(const ob_block *b, int c, const int idx[3], double t)
{
    double J = 0.0;
    for (int s = 0; s < b->nsrc; s++) {
        const ob_source *S = &b->src[s];
        if (S->comp != c) continue;
        int hit = 1;
        for (int a = 0; a < 3; a++)
            if (S->idx[a] >= 0 && S->idx[a] != idx[a]) hit = 0;
        if (hit) J += S->amp * ob_waveform(S->wf, t, S->tw, S->t0, S->f);
    }
    return J;
}

/* E^{n+1} from E^n and H^{n+1/2}, with the current density J(t^{n+1/2}):
 * eps dE/dt = curl H + SAT - J. */
static void e_half_step(ob_block *b)
{
    double dt = b->dt;
    double t = ((double)b->step + 0.5) * dt;
    for (int c = EX; c <= EZ; c++) {
        int e0 = ext(b, c, 0), e1 = ext(b, c, 1), e2 = ext(b, c, 2);
        int has_src = 0;
        for (int s = 0; s < b->nsrc; s++) if (b->src[s].comp == c) has_src = 1;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < e2; k++)
            for (int j = 0; j < e1; j++)
                for (int i = 0; i < e0; i++) {
                    int idx[3] = {i, j, k};
                    double L, g;
                    node_rhs(b, c, idx, &L, &g);
                    size_t o = at(b, c, i, j, k);
                    if (has_src) L -= source_value(b, c, idx, t) / (OB_EPS0 * b->epsn[c][o]);
                    b->rhs[c][o] = ((1.0 - 0.5 * dt * g) * b->F[c][o] + dt * L) / (1.0 + 0.5 * dt * g);
                }
    }
    /* E of this block is replaced only after all its nodes are computed;
     * other blocks read E only during the H half-step. */
    for (int c = EX; c <= EZ; c++) memcpy(b->F[c], b->rhs[c], count(b, c) * sizeof(double));
}

static void sample_probes(ob_block *b, int want_h)
{
    if (!b->prb_buf) return;
    long s = b->step;
    if (s >= b->prb_cap) return;
    for (int p = 0; p < b->nprb; p++) {
        ob_probe *P = &b->prb[p];
        if ((P->comp >= HX) != want_h) continue;
        b->prb_buf[(size_t)p * b->prb_cap + s] = b->F[P->comp][at(b, P->comp, P->idx[0], P->idx[1], P->idx[2])];
    }
}

/* nsteps leapfrog steps of all blocks together: first every block's H
 * half-step (interfaces read the neighbours' E^n), then every block's E
 * half-step (interfaces read the neighbours' H^{n+1/2}).  Probes record
 * H^{n+1/2} and E^{n+1} in slot n. */
void ob_step(ob_block **blocks, int nb, long nsteps)
{
    for (long s = 0; s < nsteps; s++) {
        for (int bi = 0; bi < nb; bi++) {
            ob_block *b = blocks[bi];
            double *dst[3] = {b->tmp[0], b->tmp[1], b->tmp[2]};
            h_half_step(b, dst);
        }
        for (int bi = 0; bi < nb; bi++) {
            ob_block *b = blocks[bi];
            for (int c = 0; c < 3; c++) memcpy(b->F[HX + c], b->tmp[c], count(b, HX + c) * sizeof(double));
            sample_probes(b, 1);
        }
        for (int bi = 0; bi < nb; bi++) e_half_step(blocks[bi]);
        for (int bi = 0; bi < nb; bi++) {
            sample_probes(blocks[bi], 0);
            blocks[bi]->step++;
        }
    }
}

/* W^n = 1/2 [ sum_E eps P''' (E^n)^2 + sum_H mu P''' H^{n-1/2} H^{n+1/2} ],
 * the discrete energy of Eq. (16) in the form conserved by leapfrog. */
double ob_energy(ob_block **blocks, int nb)
{
    for (int bi = 0; bi < nb; bi++) {
        ob_block *b = blocks[bi];
        double *dst[3] = {b->tmp[0], b->tmp[1], b->tmp[2]};
        h_half_step(b, dst);
    }
    double W = 0.0;
    for (int bi = 0; bi < nb; bi++) {
        ob_block *b = blocks[bi];
        for (int c = 0; c < 6; c++) {
            int e0 = ext(b, c, 0), e1 = ext(b, c, 1), e2 = ext(b, c, 2);
            double part = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : part)
            for (int k = 0; k < e2; k++)
                for (int j = 0; j < e1; j++)
                    for (int i = 0; i < e0; i++) {
                        size_t o = at(b, c, i, j, k);
                        double w = w1(b, c, 0, i) * w1(b, c, 1, j) * w1(b, c, 2, k);
                        if (c < HX)
                            part += OB_EPS0 * b->epsn[c][o] * w * b->F[c][o] * b->F[c][o];
                        else
                            part += OB_MU0 * b->mun[c][o] * w * b->F[c][o] * b->tmp[c - HX][o];
                    }
            W += part;
        }
    }
    return 0.5 * W;
}

void ob_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int ob_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
