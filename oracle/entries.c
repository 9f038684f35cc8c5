/*
 * ORACLE (test infrastructure only; never linked into the product library).
 *
 * Plain FP64 CPU evaluation of the Galerkin panel-pair integrals of the
 * VoxCap surface integral equations, written from the definitions:
 *
 *   P'_kl = (1/4pi) Int_{S_k} Int_{S_l} 1/|r - r'| dS' dS              (Eq. 5)
 *   E'_kl = d/dn_k  (1/4pi) Int_{S_k} Int_{S_l} 1/|r - r'| dS' dS      (Eq. 6)
 *
 * in normalised units (voxel edge 1, epsilon_0 absorbed: the physical entries
 * are these times dv^3/eps0 and dv^2/eps0, Appendix C).  n_k is the +axis unit
 * normal of the test panel k, i.e. E' is the derivative of the tested
 * potential when the test panel is translated along +n_k.
 *
 * Method (deliberately different from the GPU path, which uses 4-D corner
 * sums and Gauss-Legendre): the inner integral over the source square is the
 * closed-form potential / field of a uniformly charged rectangle (textbook
 * corner sums of asinh / atan terms, derived from the definition); the outer
 * 2-D integral over the test square is a nested, globally adaptive 15-point
 * Gauss-Kronrod quadrature.  Every singularity of the integrand (source edges
 * projected on the test square, the shared edge of touching orthogonal
 * panels) lies on the boundary of an integration interval because all panel
 * corners sit on the integer / half-integer voxel lattice.
 *
 * Special cases fixed by the definitions:
 *   - coplanar parallel panels: E' = 0 (the normal field of a flat charge in
 *     its own plane is zero; for the self term this is the principal value).
 *
 * Geometry: a panel is a unit square normal to axis `orient` (0=x,1=y,2=z),
 * given by its centre.  oracle_entry() takes the centre difference
 * d = c_test - c_source.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#define INV4PI 0.079577471545947667884441881686257181017229822870228

/* ---- inner closed forms: unit-density square [-1/2,1/2]^2 in plane z=0 ---- */

/* asinh(v2/rho) - asinh(v1/rho) for v1 < v2; rho >= 0.  For rho == 0 and
 * v1, v2 of one sign this is the limit sign*ln(|v2|/|v1|). */
static double asinh_diff(double v1, double v2, double rho)
{
    if (rho > 0.0) return asinh(v2 / rho) - asinh(v1 / rho);
    if (v1 > 0.0) return log(v2 / v1);
    if (v2 < 0.0) return log(v1 / v2);   /* |v1| / |v2| */
    return HUGE_VAL;                     /* on the charged segment: never sampled */
}

/* potential Int_sq 1/r  at (X,Y,Z) */
static double sq_pot(double X, double Y, double Z)
{
    const double xs[2] = {-0.5 - X, 0.5 - X};   /* u = x_corner - X */
    const double ys[2] = {-0.5 - Y, 0.5 - Y};   /* v = y_corner - Y */
    double s = 0.0;
    /* u * ln(v + r) summed over the corner v's = u * [asinh(v2/rho)-asinh(v1/rho)] */
    for (int a = 0; a < 2; ++a) {
        double u = xs[a];
        if (u == 0.0) continue;
        double rho = sqrt(u * u + Z * Z);
        s += (a ? 1.0 : -1.0) * u * asinh_diff(ys[0], ys[1], rho);
    }
    for (int b = 0; b < 2; ++b) {
        double v = ys[b];
        if (v == 0.0) continue;
        double rho = sqrt(v * v + Z * Z);
        s += (b ? 1.0 : -1.0) * v * asinh_diff(xs[0], xs[1], rho);
    }
    if (Z != 0.0) {
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double u = xs[a], v = ys[b];
                double r = sqrt(u * u + v * v + Z * Z);
                double sg = (a == b) ? 1.0 : -1.0;
                s -= sg * Z * atan(u * v / (Z * r));
            }
    }
    return s;
}

/* d/dZ of sq_pot (Z != 0) */
static double sq_dZ(double X, double Y, double Z)
{
    const double xs[2] = {-0.5 - X, 0.5 - X};
    const double ys[2] = {-0.5 - Y, 0.5 - Y};
    if (Z == 0.0) return 0.0;
    double s = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double u = xs[a], v = ys[b];
            double r = sqrt(u * u + v * v + Z * Z);
            double sg = (a == b) ? 1.0 : -1.0;
            s -= sg * atan(u * v / (Z * r));
        }
    return s;
}

/* d/dX of sq_pot */
static double sq_dX(double X, double Y, double Z)
{
    const double xs[2] = {-0.5 - X, 0.5 - X};
    const double ys[2] = {-0.5 - Y, 0.5 - Y};
    double s = 0.0;
    for (int a = 0; a < 2; ++a) {
        double u = xs[a];
        double rho = sqrt(u * u + Z * Z);
        s -= (a ? 1.0 : -1.0) * asinh_diff(ys[0], ys[1], rho);
    }
    return s;
}

/* d/dY of sq_pot */
static double sq_dY(double X, double Y, double Z) { return sq_dX(Y, X, Z); }

/* ---- globally adaptive Gauss-Kronrod (7/15) in 1-D ---- */

typedef double (*fn1)(double, void *);

static const double XGK[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double WGK[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double WG[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

static double gk15(fn1 f, void *ctx, double a, double b, double *err)
{
    double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double fc = f(c, ctx);
    double rk = fc * WGK[7], rg = fc * WG[3];
    for (int j = 0; j < 7; ++j) {
        double x = h * XGK[j];
        double f1 = f(c - x, ctx), f2 = f(c + x, ctx);
        rk += WGK[j] * (f1 + f2);
        if (j & 1) rg += WG[j / 2] * (f1 + f2);
    }
    *err = fabs((rk - rg) * h);
    return rk * h;
}

#define MAXSEG 4000
/* integrate f over the union of [pts[i], pts[i+1]] until the summed error
 * estimate is below max(abstol, reltol*|I|). */
static double adapt(fn1 f, void *ctx, const double *pts, int npts, double reltol, double abstol)
{
    double sa[MAXSEG], sb[MAXSEG], sv[MAXSEG], se[MAXSEG];
    int n = 0;
    double tot = 0.0, toterr = 0.0;
    for (int i = 0; i + 1 < npts; ++i) {
        if (!(pts[i + 1] > pts[i])) continue;
        sa[n] = pts[i]; sb[n] = pts[i + 1];
        sv[n] = gk15(f, ctx, sa[n], sb[n], &se[n]);
        tot += sv[n]; toterr += se[n]; ++n;
    }
    for (int it = 0; it < 100000; ++it) {
        double tol = fmax(abstol, reltol * fabs(tot));
        if (toterr <= tol || n + 1 >= MAXSEG) break;
        int k = 0;
        for (int i = 1; i < n; ++i) if (se[i] > se[k]) k = i;
        double a = sa[k], b = sb[k], m = 0.5 * (a + b);
        if (!(m > a && m < b)) break;             /* cannot split further */
        double e1, e2;
        double v1 = gk15(f, ctx, a, m, &e1);
        double v2 = gk15(f, ctx, m, b, &e2);
        tot += v1 + v2 - sv[k]; toterr += e1 + e2 - se[k];
        sb[k] = m; sv[k] = v1; se[k] = e1;
        sa[n] = m; sb[n] = b; sv[n] = v2; se[n] = e2; ++n;
    }
    /* re-sum to avoid drift of the running total */
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += sv[i];
    return s;
}

/* ---- nested outer integral over the test square ---- */

/* The test square is given in the source-local frame (source = unit square
 * centred at 0 in the plane Z = 0):
 *   mode 0: parallel, test plane Z = z0, X in [x0-1/2,x0+1/2], Y in [y0-1/2,y0+1/2]
 *   mode 1: orthogonal, test plane X = x0, Y in [y0-1/2,..], Z in [z0-1/2,..]
 * and `which` selects the integrand: 0 potential, 1 d/dX, 2 d/dY, 3 d/dZ. */
typedef struct {
    int mode, which;
    double x0, y0, z0;
    double outer;   /* current value of the outer variable */
    double rtol;
} ctx_t;

static double eval_point(const ctx_t *c, double X, double Y, double Z)
{
    switch (c->which) {
    case 0: return sq_pot(X, Y, Z);
    case 1: return sq_dX(X, Y, Z);
    case 2: return sq_dY(X, Y, Z);
    default: return sq_dZ(X, Y, Z);
    }
}

/* split points of an interval [lo,hi] at the source edges -1/2, +1/2 and 0 */
static int breakpoints(double lo, double hi, double *pts)
{
    int n = 0;
    pts[n++] = lo;
    const double cand[3] = {-0.5, 0.0, 0.5};
    for (int i = 0; i < 3; ++i)
        if (cand[i] > lo && cand[i] < hi) pts[n++] = cand[i];
    pts[n++] = hi;
    return n;
}

static double inner_fn(double t, void *vp)
{
    const ctx_t *c = (const ctx_t *)vp;
    if (c->mode == 0) return eval_point(c, c->outer, t, c->z0);   /* t = Y */
    return eval_point(c, c->x0, t, c->outer);                      /* t = Y, outer = Z */
}

static double outer_fn(double s, void *vp)
{
    ctx_t c = *(const ctx_t *)vp;
    c.outer = s;
    double pts[5];
    int n = breakpoints(c.y0 - 0.5, c.y0 + 0.5, pts);
    return adapt(inner_fn, &c, pts, n, 0.1 * c.rtol, 1e-300);
}

static double outer_integral(ctx_t *c)
{
    double pts[5];
    int n;
    if (c->mode == 0) n = breakpoints(c->x0 - 0.5, c->x0 + 0.5, pts);   /* outer over X */
    else n = breakpoints(c->z0 - 0.5, c->z0 + 0.5, pts);                /* outer over Z */
    return adapt(outer_fn, c, pts, n, c->rtol, 1e-300);
}

/*
 * oracle_entry: kind 0 -> P' (Eq. 5), kind 1 -> E' (Eq. 6), normalised units.
 * test_orient / src_orient in {0,1,2}; (dx,dy,dz) = test centre - source centre.
 */
double oracle_entry(int kind, int test_orient, int src_orient,
                    double dx, double dy, double dz, double rtol)
{
    const double d[3] = {dx, dy, dz};
    const int nb = src_orient;
    /* source-local frame: X = first in-plane axis, Y = second, Z = normal */
    int ax = (nb == 0) ? 1 : 0;
    int ay = (nb == 2) ? 1 : 2;
    ctx_t c;
    c.rtol = rtol;
    if (test_orient == src_orient) {
        c.mode = 0;
        c.x0 = d[ax]; c.y0 = d[ay]; c.z0 = d[nb];
        if (kind == 0) c.which = 0;
        else {
            if (c.z0 == 0.0) return 0.0;   /* coplanar: zero normal field */
            c.which = 3;                   /* test normal = +Z */
        }
    } else {
        /* test normal alpha is one of the source in-plane axes */
        int alpha = test_orient;
        int gamma = 3 - alpha - nb;        /* the shared in-plane axis */
        c.mode = 1;
        c.x0 = d[alpha]; c.y0 = d[gamma]; c.z0 = d[nb];
        if (kind == 0) c.which = 0;
        else c.which = 1;                  /* d/d(alpha) = d/dX in the remapped frame */
        /* Remap: in mode 1 the test square is {X = x0} x [Y] x [Z]; the source
         * square's in-plane axes are (ax, ay).  We evaluate the source fields
         * with X := alpha-coordinate and Y := gamma-coordinate; the square is
         * symmetric under swapping its in-plane axes, so this is exact. */
    }
    return INV4PI * outer_integral(&c);
}

/* batch evaluation (OpenMP over entries) */
void oracle_entries(int n, const int32_t *kind, const int32_t *to, const int32_t *so,
                    const double *dxyz, double rtol, double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n; ++i)
        out[i] = oracle_entry(kind[i], to[i], so[i], dxyz[3 * i], dxyz[3 * i + 1],
                              dxyz[3 * i + 2], rtol);
}

/* raw square potential / fields, exported so that tests can pin them
 * (e.g. against Gauss's law and finite differences) */
double oracle_square_field(int which, double X, double Y, double Z)
{
    switch (which) {
    case 0: return sq_pot(X, Y, Z);
    case 1: return sq_dX(X, Y, Z);
    case 2: return sq_dY(X, Y, Z);
    default: return sq_dZ(X, Y, Z);
    }
}
