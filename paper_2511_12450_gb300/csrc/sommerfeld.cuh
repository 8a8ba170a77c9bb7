// sommerfeld.cuh -- Sommerfeld-integral quadrature of the reaction kernels.
//
// A reaction component (Sec. 3.1, eq. fourreactions in the interface-referenced
// form of devmath.cuh) is
//   K_c(X, h_s, h_t) = (1/2pi) int_R Sigma_c(lambda) e^{i lambda X}
//                      e^{i k_{ls,y} h_s} e^{i k_{lt,y} h_t} d lambda,
// X = x_s - x_t (matvec source minus matvec target).  Sigma_c and the two
// exponentials are even in lambda, so
//   K_c = (1/pi) int_0^T (...) cos(lambda X) d lambda                (detour)
//       + (1/2pi) int_T^inf (...) e^{+i lambda X} + (...) e^{-i lambda X}   (rays)
// The detour lambda(t) = t - i h sin(pi t / T), t in [0, T], passes below the
// real-axis poles and branch points (T = 1.2 k_max + 1, h = min(1/2, 1/|X|));
// it is integrated with 8-point Gauss-Legendre panels whose number grows with
// the oscillation (|X| + D).  Past T each half is rotated onto the ray
// lambda = T + t u, u = (D_+ +- i X)/rho (D_+ = max(D, 0), rho = |D_+ + iX|),
// along which e^{+-i lambda X - lambda D} decays like e^{-rho t} without
// oscillating; the ray is integrated with the exp-sinh (double-exponential)
// rule, which resolves both the fast decay and the near-singular behaviour of
// points close to an interface.  D = h_s + h_t + H_c is the effective
// transmission distance of the pair (Sec. 3.2).
//
// The M2L moments of Sec. 4.1 (eq. generalintegral) use the same construction on
// their own contour (table_contour_node: a shorter detour that keeps its depth to
// its end, where the rays start):
//   I_{nm} = (1/2pi) int Sigma e^{i lambda X} e^{i k_a h_S} e^{i k_b h_T}
//            w(lambda,k_a)^n w(lambda,k_b)^{-m} d lambda,
// split into the two halves e^{+i lambda X} w_a^n w_b^{-m} and
// e^{-i lambda X} w_a^{-n} w_b^{m} (w(-lambda) = 1/w(lambda)).
#pragma once
#include "devmath.cuh"
#include "geometry.h"

namespace lfmm {

struct QuadNode {
    cd lam;     // node
    cd fp;      // weight multiplying the e^{+i lambda X} half (already includes e^{+i lambda X})
    cd fm;      // weight multiplying the e^{-i lambda X} half (already includes e^{-i lambda X})
};

// Panels of the detour: enough for the oscillation (|X| + D), and no wider than the
// detour's depth at the smallest branch point k_min, h sin(pi k_min / T): in media whose
// top or bottom wavenumber is small against k_max the half-sine passes close above that
// branch point (Example 2 of Sec. 5, k = 1.2 under k_max = 10: depth 0.14 under 0.48-wide
// panels lost 3e-7 on entries near the interface; at most one depth per panel keeps them
// at the rule's 1e-12 level).
__device__ __forceinline__ int detour_panels(const QuadRule& q, double X, double D, double* h_out) {
    double ax = fabs(X);
    double h = fmin(0.5, 1.0 / fmax(ax, 1e-3));
    *h_out = h;
    double need = q.T * (1.0 / h + 0.6 * (fmax(D, 0.0) + ax));
    need = fmax(need, q.T / (h * sinpi(q.kmin / q.T)));
    int P = (int)ceil(need);
    return P > q.min_panels ? P : q.min_panels;
}

// Node j of the contour for a pair with horizontal offset X and effective
// distance D: j < 8P on the detour, then nes nodes on the + ray, then nes on
// the - ray.  Returns lambda and the weights (with dlambda, 1/(2pi) and the
// oscillatory factor) of the two halves.
__device__ __forceinline__ QuadNode contour_node(const QuadRule& q, int j, int P, double h, double X, double D) {
    QuadNode out;
    const int ndet = P * 8;
    const double inv2pi = 0.15915494309189533577;
    if (j < ndet) {
        int pan = j >> 3, r = j & 7;
        double a0 = q.T * (double)pan / P, a1 = q.T * (double)(pan + 1) / P;
        double hl = 0.5 * (a1 - a0);
        double t = 0.5 * (a0 + a1) + hl * q.gl_x[r];
        double wt = hl * q.gl_w[r];
        double s, c;
        sincospi(t / q.T, &s, &c);
        out.lam = mk(t, -h * s);
        cd dl = mk(1.0, -h * (M_PI / q.T) * c);
        // e^{+i lambda X} and e^{-i lambda X}
        cd ep = cexpd(mk(-out.lam.y * X, out.lam.x * X));
        cd em = cexpd(mk(out.lam.y * X, -out.lam.x * X));
        cd base = (wt * inv2pi) * dl;
        out.fp = base * ep;
        out.fm = base * em;
        return out;
    }
    int jj = j - ndet;
    int sg = (jj < q.nes) ? 1 : -1;
    int k = (jj < q.nes) ? jj : jj - q.nes;
    double v = q.es_v0 + k * q.es_hv;
    double tt = exp(M_PI_2 * sinh(v));
    double dtt = tt * M_PI_2 * cosh(v) * q.es_hv;
    double Dp = fmax(D, 0.0);
    double rr = fmax(hypot(Dp, X), 1e-300);
    cd u = mk(Dp / rr, sg * X / rr);
    out.lam = mk(q.T, 0.0) + (tt / rr) * u;
    cd e = cexpd(mk(-sg * X * out.lam.y, sg * X * out.lam.x));
    cd f = ((dtt / rr) * inv2pi) * (e * u);
    if (sg > 0) { out.fp = f; out.fm = mk(0.0, 0.0); }
    else { out.fm = f; out.fp = mk(0.0, 0.0); }
    return out;
}

// The M2L moment tables' contour: a quarter-sine detour lambda(t) = t - i h
// sin(pi t / (2 T')), t in [0, T'], T' = q.tab_T just past the largest branch point
// (it keeps its full depth there), then the two rays from T' - i h.  The region
// between this path and the real axis right of T' holds no singularity, so the
// rays replace the rest of the real axis as before.  P panels on the detour.
__host__ __device__ __forceinline__ int table_panels(const QuadRule& q, double X, double D, double* h_out) {
    double ax = fabs(X);
    double h = fmin(0.5, 1.0 / fmax(ax, 1e-3));
    *h_out = h;
    int P = (int)ceil(q.tab_T * (1.0 / h + 0.6 * (fmax(D, 0.0) + ax)));
    return P > q.min_panels ? P : q.min_panels;
}
__device__ __forceinline__ QuadNode table_contour_node(const QuadRule& q, int j, int P, double h, double X,
                                                       double D) {
    QuadNode out;
    const int ndet = P * 8;
    const double inv2pi = 0.15915494309189533577;
    const double T = q.tab_T;
    if (j < ndet) {
        int pan = j >> 3, r = j & 7;
        double a0 = T * (double)pan / P, a1 = T * (double)(pan + 1) / P;
        double hl = 0.5 * (a1 - a0);
        double t = 0.5 * (a0 + a1) + hl * q.gl_x[r];
        double wt = hl * q.gl_w[r];
        double s, c;
        sincospi(0.5 * t / T, &s, &c);
        out.lam = mk(t, -h * s);
        cd dl = mk(1.0, -h * (0.5 * M_PI / T) * c);
        cd ep = cexpd(mk(-out.lam.y * X, out.lam.x * X));
        cd em = cexpd(mk(out.lam.y * X, -out.lam.x * X));
        cd base = (wt * inv2pi) * dl;
        out.fp = base * ep;
        out.fm = base * em;
        return out;
    }
    int jj = j - ndet;
    int sg = (jj < q.tab_nes) ? 1 : -1;
    int k = (jj < q.tab_nes) ? jj : jj - q.tab_nes;
    double v = q.tab_es_v0 + k * q.tab_es_hv;
    double tt = exp(M_PI_2 * sinh(v));
    double dtt = tt * M_PI_2 * cosh(v) * q.tab_es_hv;
    double Dp = fmax(D, 0.0);
    double rr = fmax(hypot(Dp, X), 1e-300);
    cd u = mk(Dp / rr, sg * X / rr);
    out.lam = mk(T, -h) + (tt / rr) * u;
    cd e = cexpd(mk(-sg * X * out.lam.y, sg * X * out.lam.x));
    cd f = ((dtt / rr) * inv2pi) * (e * u);
    if (sg > 0) { out.fp = f; out.fm = mk(0.0, 0.0); }
    else { out.fm = f; out.fp = mk(0.0, 0.0); }
    return out;
}

__device__ __forceinline__ cd warp_sum(cd v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Reaction kernel value K_c(X, h_s, h_t); all 32 lanes of the warp must call
// it with the same arguments; every lane receives the result.
__device__ inline cd react_kernel_warp(const MediumDev& m, const QuadRule& q, int ls, int a, int lt, int b,
                                       double Hc, double X, double hs, double ht) {
    const int lane = threadIdx.x & 31;
    double D = hs + ht + Hc;
    double h;
    int P = detour_panels(q, X, D, &h);
    int ntot = P * 8 + 2 * q.nes;
    cd acc = mk(0.0, 0.0);
    for (int j = lane; j < ntot; j += 32) {
        QuadNode nd = contour_node(q, j, P, h, X, D);
        cd S = sigma_comp(m, nd.lam, ls, a, lt, b);
        cd E = eikh(ky_of(m.k[ls], nd.lam), hs) * eikh(ky_of(m.k[lt], nd.lam), ht);
        acc += (S * E) * (nd.fp + nd.fm);
    }
    return warp_sum(acc);
}

// The kernel and its derivatives with respect to the matvec source point, for the
// combined-field (double-layer) entries: d/dX multiplies the e^{+-i lambda X}
// halves by +-i lambda, d/dh_s the integrand by i k_{ls,y}.  out = {K_c, dK_c/dX,
// dK_c/dh_s}; all 32 lanes call it with the same arguments and receive the result.
__device__ inline void react_kernel_grad_warp(const MediumDev& m, const QuadRule& q, int ls, int a, int lt, int b,
                                              double Hc, double X, double hs, double ht, cd out[3]) {
    const int lane = threadIdx.x & 31;
    double D = hs + ht + Hc;
    double h;
    int P = detour_panels(q, X, D, &h);
    int ntot = P * 8 + 2 * q.nes;
    cd a0 = mk(0.0, 0.0), ax = mk(0.0, 0.0), ah = mk(0.0, 0.0);
    for (int j = lane; j < ntot; j += 32) {
        QuadNode nd = contour_node(q, j, P, h, X, D);
        cd S = sigma_comp(m, nd.lam, ls, a, lt, b);
        const cd ks = ky_of(m.k[ls], nd.lam);
        cd SE = S * (eikh(ks, hs) * eikh(ky_of(m.k[lt], nd.lam), ht));
        const cd wsum = nd.fp + nd.fm, wdif = nd.fp - nd.fm;
        a0 += SE * wsum;
        ax += (SE * mk(-nd.lam.y, nd.lam.x)) * wdif;
        ah += (SE * mk(-ks.y, ks.x)) * wsum;
    }
    out[0] = warp_sum(a0);
    out[1] = warp_sum(ax);
    out[2] = warp_sum(ah);
}

// Combined-field reaction entry (without the weight |Gamma_e|): the double layer
// n_e . grad_{c_e} K_c plus -i k_ls K_c.  The source height h_s grows with y when
// it is measured from the layer's bottom (a = 0) and shrinks when from its top.
__device__ __forceinline__ cd react_cf_combine(const cd g[3], int a, double kls, double nx, double ny) {
    const double sy = (a == 0) ? ny : -ny;
    return mk(nx * g[1].x + sy * g[2].x + kls * g[0].y, nx * g[1].y + sy * g[2].y - kls * g[0].x);
}

}  // namespace lfmm
