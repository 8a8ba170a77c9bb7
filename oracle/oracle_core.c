/*
 * oracle_core.c -- plain FP64 CPU reference for the layered-medium reaction
 * Green's function.  TEST INFRASTRUCTURE ONLY: used by tests/, by the smoke
 * check and by the CPU-baseline leg of bench.py; the product path never calls
 * it.
 *
 * What it computes (paper Sec. 3.1):
 *   G_{ll'}(r, r') = delta_{ll'} G^f_l(r, r') + G^r_{ll'}(r, r')      (eq. layeredGreensfun)
 *   G^r_{ll'}(r, r') = (1/2pi) int_R  Gt^r(lambda; y, y') e^{i lambda (x-x')} d lambda
 * where Gt^r is the spectral reaction field of a unit line source at y' in
 * layer l', observed at y in layer l.
 *
 * Gt^r is obtained here by a DIRECT interface solve, deliberately not by the
 * paper's reflection/transmission recursions (eqs. Rellrecursionup,
 * Rellrecursiondown, generaltransmission and the densities of Cases I-III), so
 * that those recursions can be checked against it.  In every layer m the field
 * is written as
 *     a_m e^{i k_m (y + d_m)}  +  b_m e^{i k_m (-d_{m-1} - y)}
 * (up-going wave referenced at the layer's bottom interface, down-going wave at
 * its top interface), plus the free wave (i/(2k')) e^{i k' |y-y'|} in the
 * source layer.  Every exponential has modulus <= 1 inside its layer.  The top
 * layer has no b_0 and the bottom layer no a_L (outgoing conditions); the
 * transmission conditions [G] = 0 and [eta dG/dy] = 0 at the L interfaces (the
 * interface conditions of Sec. 3.1) give a 2L x 2L system, solved by Gaussian
 * elimination with partial pivoting.  The branch of k_y = sqrt(k^2 - lambda^2)
 * is the one with Im k_y >= 0.
 *
 * The right-hand side depends on y' only through e^{i k' h_up(y')} and
 * e^{i k' h_dn(y')} (the free wave's values at the top and bottom interfaces
 * of the source layer), so solving with the two unit excitations gives the
 * four amplitudes of the reaction field (field arriving up/down x source
 * leaving up/down).
 *
 * The lambda integral is taken along a deformed contour:
 *   * [0, T], T = 1.2 max k + 1: lambda(t) = t - i h sin(pi t/T), a detour
 *     into the fourth quadrant that passes below the real-axis poles and the
 *     branch points; h = min(1/2, 1/|X|) so that cos(lambda X) grows by at most
 *     cosh(1).  Integrand (1/pi) Gt^r cos(lambda X) (Gt^r is even in lambda).
 *   * [T, inf): cos = (e^{i lambda X} + e^{-i lambda X})/2, each half rotated
 *     onto the ray lambda = T + t u with u = (D +- iX)/rho, rho = sqrt(X^2+D^2),
 *     D the smallest vertical travel distance of the reflected waves; along it
 *     e^{+-i lambda X} e^{-lambda D} decays like e^{-rho t} without oscillating
 *     (Jordan's lemma: no singularity lies in the swept sector).
 * Gradient with respect to the FIELD point (x, y), for the double-layer
 * (combined-field) kernel: d/dx multiplies the spectral integrand by i lambda
 * (cos(lambda X) becomes -lambda sin(lambda X) on the detour, e^{+-i lambda X}
 * gains +-i lambda on the rays); d/dy multiplies the wave arriving from below
 * (referenced at the field layer's bottom, e^{i k_y (y + d)}) by +i k_y and the
 * wave arriving from above (e^{i k_y (-d' - y)}) by -i k_y.
 * Both pieces use adaptive Gauss-Kronrod (7,15) quadrature (Kronrod 1965;
 * the node/weight values are the standard published ones), the ray after the
 * map t = s/((1-s) rho), s in [0,1).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define MAXLAY 16

typedef struct {
    int nl;                /* number of layers L+1 */
    double yint[MAXLAY];   /* interface heights y_j = -d_j, j = 0..L-1, decreasing */
    double k[MAXLAY];      /* real wavenumbers */
    double eta[MAXLAY];    /* densities */
} medium_t;

static const double PI = 3.14159265358979323846264338327950288;

/* ---- Gauss-Kronrod (7,15): abscissae and weights on [-1,1] ---------------- */
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

/* ---- helpers ---------------------------------------------------------------- */

/* k_y with Im k_y >= 0 */
static cplx ky_of(double k, cplx lam) {
    cplx s = csqrt(k * k - lam * lam);
    if (cimag(s) < 0.0) s = -s;
    return s;
}

static double thick(const medium_t *m, int l) { /* thickness of an interior layer */
    return m->yint[l - 1] - m->yint[l];
}

/* Solve A x = B (n x n, nrhs columns, column-major B), partial pivoting.
 * Returns 0 on success, -1 if singular. */
static int gauss_solve(int n, cplx *A, int nrhs, cplx *B) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = cabs(A[c * n + c]);
        for (int r = c + 1; r < n; ++r) {
            double v = cabs(A[r * n + c]);
            if (v > best) { best = v; piv = r; }
        }
        if (best == 0.0) return -1;
        if (piv != c) {
            for (int j = 0; j < n; ++j) { cplx t = A[c * n + j]; A[c * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
            for (int q = 0; q < nrhs; ++q) { cplx t = B[q * n + c]; B[q * n + c] = B[q * n + piv]; B[q * n + piv] = t; }
        }
        cplx inv = 1.0 / A[c * n + c];
        for (int r = c + 1; r < n; ++r) {
            cplx f = A[r * n + c] * inv;
            if (f == 0.0) continue;
            for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
            for (int q = 0; q < nrhs; ++q) B[q * n + r] -= f * B[q * n + c];
        }
    }
    for (int q = 0; q < nrhs; ++q) {
        for (int r = n - 1; r >= 0; --r) {
            cplx s = B[q * n + r];
            for (int j = r + 1; j < n; ++j) s -= A[r * n + j] * B[q * n + j];
            B[q * n + r] = s / A[r * n + r];
        }
    }
    return 0;
}

/*
 * Spectral reaction amplitudes for field layer lf and source layer ls at
 * (complex) lambda.  S[0]: field up / source up, S[1]: field up / source down,
 * S[2]: field down / source up, S[3]: field down / source down.  Amplitudes of
 * terms that cannot exist are set to 0.  Returns 0 on success.
 */
static int spectral_amp(const medium_t *m, cplx lam, int lf, int ls, cplx S[4]) {
    int L = m->nl - 1;
    S[0] = S[1] = S[2] = S[3] = 0.0;
    if (L == 0) return 0;
    int n = 2 * L;
    cplx A[4 * MAXLAY * MAXLAY];
    cplx B[2 * 2 * MAXLAY];
    cplx kyv[MAXLAY], ev[MAXLAY];
    memset(A, 0, sizeof(cplx) * n * n);
    memset(B, 0, sizeof(cplx) * 2 * n);
    for (int l = 0; l <= L; ++l) {
        kyv[l] = ky_of(m->k[l], lam);
        ev[l] = (l >= 1 && l <= L - 1) ? cexp(I * kyv[l] * thick(m, l)) : 0.0;
    }
    /* unknown indices: a_l -> l (l = 0..L-1), b_l -> L + l - 1 (l = 1..L) */
#define IA(l) (l)
#define IB(l) (L + (l) - 1)
    for (int j = 0; j < L; ++j) {
        int rc = 2 * j, rf = 2 * j + 1;
        int up = j, lo = j + 1; /* layer above and below interface j */
        /* layer above: a_up * 1 + b_up * e_up */
        A[rc * n + IA(up)] += 1.0;
        A[rf * n + IA(up)] += m->eta[up] * I * kyv[up];
        if (up >= 1) {
            A[rc * n + IB(up)] += ev[up];
            A[rf * n + IB(up)] += -m->eta[up] * I * kyv[up] * ev[up];
        }
        /* layer below (subtracted): a_lo * e_lo + b_lo * 1 */
        if (lo <= L - 1) {
            A[rc * n + IA(lo)] -= ev[lo];
            A[rf * n + IA(lo)] -= m->eta[lo] * I * kyv[lo] * ev[lo];
        }
        A[rc * n + IB(lo)] -= 1.0;
        A[rf * n + IB(lo)] -= -m->eta[lo] * I * kyv[lo];
        /* source terms moved to the right-hand side.
         * column 0: unit "up" excitation (free wave leaving the source upward,
         *           value (i/2k') at the top interface of layer ls);
         * column 1: unit "down" excitation (value (i/2k') at the bottom interface). */
        cplx ks = kyv[ls];
        if (lo == ls) {            /* interface j is the top of the source layer */
            B[0 * n + rc] += I / (2.0 * ks);
            B[0 * n + rf] += -m->eta[lo] * 0.5;
        }
        if (up == ls) {            /* interface j is the bottom of the source layer */
            B[1 * n + rc] += -I / (2.0 * ks);
            B[1 * n + rf] += -m->eta[up] * 0.5;
        }
    }
    if (gauss_solve(n, A, 2, B) != 0) return -1;
    int has_up_src = (ls >= 1), has_dn_src = (ls <= L - 1);
    int has_up_fld = (lf <= L - 1), has_dn_fld = (lf >= 1);
    if (has_up_fld && has_up_src) S[0] = B[0 * n + IA(lf)];
    if (has_up_fld && has_dn_src) S[1] = B[1 * n + IA(lf)];
    if (has_dn_fld && has_up_src) S[2] = B[0 * n + IB(lf)];
    if (has_dn_fld && has_dn_src) S[3] = B[1 * n + IB(lf)];
#undef IA
#undef IB
    return 0;
}

/* distance of y (in layer l) above its bottom interface / below its top one */
static double h_above_bottom(const medium_t *m, int l, double y) { return y - m->yint[l]; }
static double h_below_top(const medium_t *m, int l, double y) { return m->yint[l - 1] - y; }

/* spectral reaction field Gt^r(lambda; y, y') */
typedef struct {
    const medium_t *m;
    int lf, ls;
    double y, ys, X, D;
    double hf_up, hf_dn, hs_up, hs_dn; /* heights (valid where the term exists) */
    int mode;                          /* 0: G^r, 1: dG^r/dx, 2: dG^r/dy (field point) */
    int err;
} pair_ctx;

static cplx gt_r(pair_ctx *c, cplx lam) {
    cplx S[4];
    if (spectral_amp(c->m, lam, c->lf, c->ls, S) != 0) { c->err = 1; return 0.0; }
    cplx kf = ky_of(c->m->k[c->lf], lam), ks = ky_of(c->m->k[c->ls], lam);
    cplx ef_up = (S[0] != 0.0 || S[1] != 0.0) ? cexp(I * kf * c->hf_up) : 0.0;
    cplx ef_dn = (S[2] != 0.0 || S[3] != 0.0) ? cexp(I * kf * c->hf_dn) : 0.0;
    cplx es_up = (S[0] != 0.0 || S[2] != 0.0) ? cexp(I * ks * c->hs_up) : 0.0;
    cplx es_dn = (S[1] != 0.0 || S[3] != 0.0) ? cexp(I * ks * c->hs_dn) : 0.0;
    cplx up = S[0] * ef_up * es_up + S[1] * ef_up * es_dn;   /* arriving from below */
    cplx dn = S[2] * ef_dn * es_up + S[3] * ef_dn * es_dn;   /* arriving from above */
    if (c->mode == 2) return I * kf * (up - dn);
    return up + dn;
}

/* integrand pieces */
typedef struct {
    pair_ctx *pc;
    int kind;      /* 0: detour on [0,T]; 1: ray with e^{+i lam X}; 2: ray with e^{-i lam X} */
    double T, h;
    cplx u;        /* ray direction */
    double rho;
} integ_ctx;

static cplx integrand(integ_ctx *ic, double s) {
    pair_ctx *pc = ic->pc;
    if (ic->kind == 0) {
        double t = s;
        cplx lam = t - I * ic->h * sin(PI * t / ic->T);
        cplx dlam = 1.0 - I * ic->h * (PI / ic->T) * cos(PI * t / ic->T);
        cplx osc = (pc->mode == 1) ? -lam * csin(lam * pc->X) : ccos(lam * pc->X);
        return gt_r(pc, lam) * osc * dlam / PI;
    }
    if (s >= 1.0) return 0.0;
    double t = s / ((1.0 - s) * ic->rho);
    double dt = 1.0 / ((1.0 - s) * (1.0 - s) * ic->rho);
    cplx lam = ic->T + t * ic->u;
    double sg = (ic->kind == 1) ? 1.0 : -1.0;
    cplx v = gt_r(pc, lam) * cexp(I * sg * lam * pc->X) * ic->u * dt / (2.0 * PI);
    if (pc->mode == 1) v *= I * sg * lam;
    return v;
}

static void gk15(integ_ctx *ic, double a, double b, cplx *res, double *err) {
    double c = 0.5 * (a + b), hl = 0.5 * (b - a);
    cplx fc = integrand(ic, c);
    cplx rk = fc * WGK[7], rg = fc * WG[3];
    for (int j = 0; j < 7; ++j) {
        double dx = hl * XGK[j];
        cplx f1 = integrand(ic, c - dx), f2 = integrand(ic, c + dx);
        rk += WGK[j] * (f1 + f2);
        if (j % 2 == 1) rg += WG[j / 2] * (f1 + f2);
    }
    *res = rk * hl;
    *err = cabs((rk - rg) * hl);
}

/* globally adaptive GK15: bisect the interval with the largest error estimate */
#define MAXSEG 4000
static cplx adapt(integ_ctx *ic, double a, double b, double tol_abs, double tol_rel, int *fail) {
    static __thread double sa[MAXSEG], sb[MAXSEG], se[MAXSEG];
    static __thread cplx sr[MAXSEG];
    int ns = 1;
    sa[0] = a; sb[0] = b;
    gk15(ic, a, b, &sr[0], &se[0]);
    for (;;) {
        cplx tot = 0.0; double etot = 0.0; int worst = 0;
        for (int i = 0; i < ns; ++i) {
            tot += sr[i]; etot += se[i];
            if (se[i] > se[worst]) worst = i;
        }
        if (etot <= tol_abs || etot <= tol_rel * cabs(tot)) return tot;
        if (ns + 1 >= MAXSEG) { *fail = 1; return tot; }
        double m = 0.5 * (sa[worst] + sb[worst]);
        sa[ns] = m; sb[ns] = sb[worst];
        sb[worst] = m;
        gk15(ic, sa[worst], sb[worst], &sr[worst], &se[worst]);
        gk15(ic, sa[ns], sb[ns], &sr[ns], &se[ns]);
        ++ns;
    }
}

static int layer_of(const medium_t *m, double y) {
    int l = 0;
    while (l < m->nl - 1 && y < m->yint[l]) ++l;
    return l;
}

/*
 * G^r_{lf,ls}((x,y),(xs,ys)) for one pair.  Returns 0 on success,
 * 1 if the quadrature did not reach tolerance, 2 on a degenerate pair
 * (a point on an interface), 3 on a singular interface system.
 */
static int gr_pair_contour(const medium_t *m, double x, double y, double xs, double ys,
                           double tol_rel, int mode, double t_scale, double h_scale, cplx *out) {
    *out = 0.0;
    int L = m->nl - 1;
    if (L == 0) return 0;
    pair_ctx pc;
    memset(&pc, 0, sizeof(pc));
    pc.m = m;
    pc.mode = mode;
    pc.lf = layer_of(m, y);
    pc.ls = layer_of(m, ys);
    pc.y = y; pc.ys = ys; pc.X = x - xs;
    if (pc.lf <= L - 1) pc.hf_up = h_above_bottom(m, pc.lf, y);
    if (pc.lf >= 1) pc.hf_dn = h_below_top(m, pc.lf, y);
    if (pc.ls >= 1) pc.hs_up = h_below_top(m, pc.ls, ys);
    if (pc.ls <= L - 1) pc.hs_dn = h_above_bottom(m, pc.ls, ys);
    /* smallest vertical distance travelled by a reflected/transmitted wave */
    double D;
    if (pc.lf == pc.ls) {
        D = INFINITY;
        if (pc.ls <= L - 1) D = fmin(D, pc.hf_up + pc.hs_dn);   /* bounce off the bottom */
        if (pc.ls >= 1) D = fmin(D, pc.hf_dn + pc.hs_up);       /* bounce off the top */
    } else {
        D = fabs(y - ys);
    }
    if (!(D > 0.0)) return 2;
    pc.D = D;
    double kmax = 0.0;
    for (int l = 0; l <= L; ++l) kmax = fmax(kmax, m->k[l]);
    double T = (1.2 * kmax + 1.0) * t_scale;
    double ax = fabs(pc.X);
    double h = fmin(0.5, 1.0 / fmax(ax, 1e-3)) * h_scale;
    double rho = sqrt(pc.X * pc.X + D * D);
    int fail = 0;
    const double tol_abs = 1e-15;
    integ_ctx ic0 = {&pc, 0, T, h, 0.0, rho};
    cplx v = adapt(&ic0, 0.0, T, tol_abs, tol_rel, &fail);
    integ_ctx ic1 = {&pc, 1, T, h, (D + I * pc.X) / rho, rho};
    v += adapt(&ic1, 0.0, 1.0, tol_abs, tol_rel, &fail);
    integ_ctx ic2 = {&pc, 2, T, h, (D - I * pc.X) / rho, rho};
    v += adapt(&ic2, 0.0, 1.0, tol_abs, tol_rel, &fail);
    *out = v;
    if (pc.err) return 3;
    return fail ? 1 : 0;
}

static int gr_pair(const medium_t *m, double x, double y, double xs, double ys,
                   double tol_rel, int mode, cplx *out) {
    return gr_pair_contour(m, x, y, xs, ys, tol_rel, mode, 1.0, 1.0, out);
}

/* ---------------------------------------------------------------------------- */
/* exported entry points (called through ctypes by oracle/*.py)                 */
/* ---------------------------------------------------------------------------- */

static int make_medium(medium_t *m, int nl, const double *yint, const double *k, const double *eta) {
    if (nl < 1 || nl > MAXLAY) return -1;
    memset(m, 0, sizeof(*m));
    m->nl = nl;
    for (int j = 0; j < nl - 1; ++j) m->yint[j] = yint[j];
    for (int l = 0; l < nl; ++l) { m->k[l] = k[l]; m->eta[l] = eta[l]; }
    return 0;
}

/* Spectral amplitudes at complex lambdas: out is (n, 4) complex interleaved. */
int oracle_spectral_amp(int nl, const double *yint, const double *k, const double *eta,
                        int lf, int ls, long n, const double *lam_ri, double *out_ri) {
    medium_t m;
    if (make_medium(&m, nl, yint, k, eta)) return -1;
    for (long i = 0; i < n; ++i) {
        cplx S[4];
        cplx lam = lam_ri[2 * i] + I * lam_ri[2 * i + 1];
        if (spectral_amp(&m, lam, lf, ls, S) != 0) return -3;
        for (int q = 0; q < 4; ++q) { out_ri[8 * i + 2 * q] = creal(S[q]); out_ri[8 * i + 2 * q + 1] = cimag(S[q]); }
    }
    return 0;
}

/* G^r for n pairs: field points (x,y), source points (xs,ys).  out: complex
 * interleaved (2n).  status: per-pair status (see gr_pair). */
int oracle_gr_pairs(int nl, const double *yint, const double *k, const double *eta,
                    long n, const double *x, const double *y, const double *xs, const double *ys,
                    double tol_rel, double *out_ri, int *status) {
    medium_t m;
    if (make_medium(&m, nl, yint, k, eta)) return -1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (long i = 0; i < n; ++i) {
        cplx v;
        int st = gr_pair(&m, x[i], y[i], xs[i], ys[i], tol_rel, 0, &v);
        out_ri[2 * i] = creal(v);
        out_ri[2 * i + 1] = cimag(v);
        if (status) status[i] = st;
        if (st != 0) bad = 1;
    }
    return bad;
}

/* As oracle_gr_pairs on a contour whose detour end T is scaled by t_scale and
 * whose depth h by h_scale (both 1 for the default contour).  By Cauchy's theorem
 * the integral does not depend on the contour, so any admissible scales must
 * reproduce the default values to the quadrature tolerance: a self-check of the
 * contour and the quadrature. */
int oracle_gr_pairs_contour(int nl, const double *yint, const double *k, const double *eta,
                            long n, const double *x, const double *y, const double *xs, const double *ys,
                            double tol_rel, double t_scale, double h_scale, double *out_ri, int *status) {
    medium_t m;
    if (make_medium(&m, nl, yint, k, eta)) return -1;
    if (!(t_scale >= 1.0) || !(h_scale > 0.0 && h_scale <= 1.0)) return -1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (long i = 0; i < n; ++i) {
        cplx v;
        int st = gr_pair_contour(&m, x[i], y[i], xs[i], ys[i], tol_rel, 0, t_scale, h_scale, &v);
        out_ri[2 * i] = creal(v);
        out_ri[2 * i + 1] = cimag(v);
        if (status) status[i] = st;
        if (st != 0) bad = 1;
    }
    return bad;
}

/* Dense block of G^r: rows = field points (nr), columns = source points (nc);
 * out is row-major (nr, nc) complex interleaved. */
static int gr_block_mode(int nl, const double *yint, const double *k, const double *eta,
                         long nr, const double *xr, const double *yr,
                         long nc, const double *xc, const double *yc,
                         double tol_rel, int mode, double *out_ri) {
    medium_t m;
    if (make_medium(&m, nl, yint, k, eta)) return -1;
    int bad = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 64) reduction(| : bad)
    for (long i = 0; i < nr; ++i) {
        for (long j = 0; j < nc; ++j) {
            cplx v;
            int st = gr_pair(&m, xr[i], yr[i], xc[j], yc[j], tol_rel, mode, &v);
            out_ri[2 * (i * nc + j)] = creal(v);
            out_ri[2 * (i * nc + j) + 1] = cimag(v);
            if (st != 0) bad = 1;
        }
    }
    return bad;
}

int oracle_gr_block(int nl, const double *yint, const double *k, const double *eta,
                    long nr, const double *xr, const double *yr,
                    long nc, const double *xc, const double *yc,
                    double tol_rel, double *out_ri) {
    return gr_block_mode(nl, yint, k, eta, nr, xr, yr, nc, xc, yc, tol_rel, 0, out_ri);
}

/* Gradient of G^r with respect to the field point: out_dx, out_dy as in
 * oracle_gr_block (rows = field points, columns = source points). */
int oracle_gr_grad_block(int nl, const double *yint, const double *k, const double *eta,
                         long nr, const double *xr, const double *yr,
                         long nc, const double *xc, const double *yc,
                         double tol_rel, double *out_dx, double *out_dy) {
    int a = gr_block_mode(nl, yint, k, eta, nr, xr, yr, nc, xc, yc, tol_rel, 1, out_dx);
    int b = gr_block_mode(nl, yint, k, eta, nr, xr, yr, nc, xc, yc, tol_rel, 2, out_dy);
    return a | b;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
