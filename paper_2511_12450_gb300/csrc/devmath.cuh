// devmath.cuh -- complex FP64 helpers, Bessel recurrences and the layered-medium
// spectral densities used by every kernel of the library.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#define LFMM_MAXLAY 16

struct cd {
    double x, y;
};

__host__ __device__ __forceinline__ cd mk(double a, double b) { cd r; r.x = a; r.y = b; return r; }
__host__ __device__ __forceinline__ cd operator+(cd a, cd b) { return mk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cd operator-(cd a, cd b) { return mk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cd operator-(cd a) { return mk(-a.x, -a.y); }
__host__ __device__ __forceinline__ cd operator*(cd a, cd b) {
    return mk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ cd operator*(double s, cd a) { return mk(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ cd operator*(cd a, double s) { return mk(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ cd& operator+=(cd& a, cd b) { a.x += b.x; a.y += b.y; return a; }
__host__ __device__ __forceinline__ cd conjc(cd a) { return mk(a.x, -a.y); }
#ifdef __CUDACC__
// x or -x (neg odd) and v or -v by flipping sign bits with integer instructions: a
// conditional negation of a double otherwise costs an instruction on the FP64 pipe,
// which bounds the expansion kernels
__device__ __forceinline__ double dsign(double x, int neg) {
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)(neg & 1) << 63));
}
__device__ __forceinline__ cd csign(cd v, int neg) { return mk(dsign(v.x, neg), dsign(v.y, neg)); }
#endif
__host__ __device__ __forceinline__ double absc(cd a) { return hypot(a.x, a.y); }
__host__ __device__ __forceinline__ cd cdiv(cd a, cd b) {
    // scaled division (Smith's method)
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return mk((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.x * r + b.y;
        return mk((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__host__ __device__ __forceinline__ cd cinv(cd b) { return cdiv(mk(1.0, 0.0), b); }
// A complex value with its own binary exponent, m 2^e (max(|m.x|, |m.y|) in [0.5, 1), or
// m = 0): products of many factors without intermediate overflow or underflow.  The
// rescaling is by powers of two, so a product rounds as the plain one does wherever that
// stays in range.
struct xcd {
    cd m;
    int e;
};
__host__ __device__ __forceinline__ xcd xnorm(cd m, int e) {
    const double a = fmax(fabs(m.x), fabs(m.y));
    xcd r;
    if (!(a > 0.0) || !(a <= 1.7e308)) { r.m = m; r.e = e; return r; }   // zero or not finite: as is
    int k = 0;
    frexp(a, &k);
    r.m.x = ldexp(m.x, -k);
    r.m.y = ldexp(m.y, -k);
    r.e = e + k;
    return r;
}
__host__ __device__ __forceinline__ xcd xmul(xcd a, xcd b) {
    cd m;
    m.x = a.m.x * b.m.x - a.m.y * b.m.y;
    m.y = a.m.x * b.m.y + a.m.y * b.m.x;
    return xnorm(m, a.e + b.e);
}
// the plain value (0 below the smallest double, infinite above the largest)
__host__ __device__ __forceinline__ cd xval(xcd a) {
    cd r;
    r.x = ldexp(a.m.x, a.e);
    r.y = ldexp(a.m.y, a.e);
    return r;
}
// f u^k (k of either sign) by binary exponentiation on scaled values
__host__ __device__ __forceinline__ xcd xpow_times(cd f, cd u, int k) {
    xcd bb;
    bb = xnorm(k >= 0 ? u : cinv(u), 0);
    xcd cur = xnorm(f, 0);
    for (int k2 = k >= 0 ? k : -k; k2 > 0; k2 >>= 1) {
        if (k2 & 1) cur = xmul(cur, bb);
        if (k2 > 1) bb = xmul(bb, bb);
    }
    return cur;
}
// fused a += b * c
__host__ __device__ __forceinline__ void cfma(cd& a, cd b, cd c) {
    a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
    a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}
__host__ __device__ __forceinline__ cd cexpd(cd z) {
    double s, c;
    sincos(z.y, &s, &c);
    double e = exp(z.x);
    return mk(e * c, e * s);
}
// principal square root
__host__ __device__ __forceinline__ cd csqrtd(cd z) {
    double a = z.x, b = z.y;
    if (a == 0.0 && b == 0.0) return mk(0.0, 0.0);
    double r = hypot(a, b);
    if (a >= 0.0) {
        double t = sqrt(0.5 * (r + a));
        return mk(t, b / (2.0 * t));
    }
    double t = sqrt(0.5 * (r - a));
    return mk(fabs(b) / (2.0 * t), copysign(t, b));
}
// k_y = sqrt(k^2 - lambda^2) on the sheet Im k_y >= 0 (outgoing/decaying)
__host__ __device__ __forceinline__ cd ky_of(double k, cd lam) {
    cd l2 = lam * lam;
    cd s = csqrtd(mk(k * k - l2.x, -l2.y));
    if (s.y < 0.0) s = -s;
    return s;
}
// w(lambda, k) = (k_y + i lambda) / k   (Sec. 4.1, Proposition)
__host__ __device__ __forceinline__ cd w_of(cd kyv, cd lam, double k) {
    return mk((kyv.x - lam.y) / k, (kyv.y + lam.x) / k);
}

// ---------------------------------------------------------------------------
// Bessel functions J_0..J_p(x), x >= 0, by Miller's backward recurrence
// normalised with J_0 + 2 sum_k J_2k = 1 (Abramowitz & Stegun 9.12; the
// "Miller algorithm").  `out` must hold p+1 doubles.
// ---------------------------------------------------------------------------
__host__ __device__ inline void bessel_j_seq(double x, int p, double* out) {
    if (x < 1e-300) {
        out[0] = 1.0;
        for (int n = 1; n <= p; ++n) out[n] = 0.0;
        return;
    }
    const int m = (p > (int)x) ? p : (int)x;
    int start = m + 16 + (int)(3.0 * sqrt((double)m));
    if (start & 1) ++start;
    const double tx = 2.0 / x;
    double jp1 = 0.0, j = 1e-280, norm = 0.0;
    // walk down from start to 0; store entries n <= p
    for (int n = start; n >= 0; --n) {
        if (n <= p) out[n] = j;
        if ((n & 1) == 0) norm += (n == 0 ? j : 2.0 * j);
        double jm1 = (n > 0) ? (n * tx) * j - jp1 : 0.0;
        jp1 = j;
        j = jm1;
        if (fabs(j) > 1e250) {  // rescale to avoid overflow
            const double sc = 1e-250;
            j *= sc; jp1 *= sc; norm *= sc;
            for (int q = n; q <= p; ++q) if (q >= 0) out[q] *= sc;
        }
    }
    const double inv = 1.0 / norm;
    for (int n = 0; n <= p; ++n) out[n] *= inv;
}

// 1/i for i = 0..127 (0 at i = 0): reciprocals as multiplications, since an FP64
// division costs a dozen FP64-pipe instructions
static __device__ const double k_inv_int[128] = {0.0,1.0 / 1,1.0 / 2,1.0 / 3,1.0 / 4,1.0 / 5,1.0 / 6,1.0 / 7,1.0 / 8,1.0 / 9,1.0 / 10,1.0 / 11,1.0 / 12,1.0 / 13,1.0 / 14,1.0 / 15,1.0 / 16,1.0 / 17,1.0 / 18,1.0 / 19,1.0 / 20,1.0 / 21,1.0 / 22,1.0 / 23,1.0 / 24,1.0 / 25,1.0 / 26,1.0 / 27,1.0 / 28,1.0 / 29,1.0 / 30,1.0 / 31,1.0 / 32,1.0 / 33,1.0 / 34,1.0 / 35,1.0 / 36,1.0 / 37,1.0 / 38,1.0 / 39,1.0 / 40,1.0 / 41,1.0 / 42,1.0 / 43,1.0 / 44,1.0 / 45,1.0 / 46,1.0 / 47,1.0 / 48,1.0 / 49,1.0 / 50,1.0 / 51,1.0 / 52,1.0 / 53,1.0 / 54,1.0 / 55,1.0 / 56,1.0 / 57,1.0 / 58,1.0 / 59,1.0 / 60,1.0 / 61,1.0 / 62,1.0 / 63,1.0 / 64,1.0 / 65,1.0 / 66,1.0 / 67,1.0 / 68,1.0 / 69,1.0 / 70,1.0 / 71,1.0 / 72,1.0 / 73,1.0 / 74,1.0 / 75,1.0 / 76,1.0 / 77,1.0 / 78,1.0 / 79,1.0 / 80,1.0 / 81,1.0 / 82,1.0 / 83,1.0 / 84,1.0 / 85,1.0 / 86,1.0 / 87,1.0 / 88,1.0 / 89,1.0 / 90,1.0 / 91,1.0 / 92,1.0 / 93,1.0 / 94,1.0 / 95,1.0 / 96,1.0 / 97,1.0 / 98,1.0 / 99,1.0 / 100,1.0 / 101,1.0 / 102,1.0 / 103,1.0 / 104,1.0 / 105,1.0 / 106,1.0 / 107,1.0 / 108,1.0 / 109,1.0 / 110,1.0 / 111,1.0 / 112,1.0 / 113,1.0 / 114,1.0 / 115,1.0 / 116,1.0 / 117,1.0 / 118,1.0 / 119,1.0 / 120,1.0 / 121,1.0 / 122,1.0 / 123,1.0 / 124,1.0 / 125,1.0 / 126,1.0 / 127};

// J_0..J_p(x) where x is small against the order (x < p / 4, p <= 80): J_p and
// J_{p-1} from the power series J_n(x) = (x/2)^n / n! sum_k (-x^2/4)^k / (k! (n+1)...(n+k))
// (A&S 9.1.10; a few terms there), then the three-term recurrence downward,
// J_{n-1} = (2n/x) J_n - J_{n+1}, which is stable in that direction for the
// minimal solution J_n and needs no normalisation.  Elsewhere Miller's algorithm;
// where (x/2)^p underflows, the two leading series terms.  Device only (uses the
// reciprocal table).
__device__ inline void bessel_j_seq_small(double x, int p, double* out) {
    if (!(x < 0.25 * p) || p < 2 || p > 80) { bessel_j_seq(x, p, out); return; }
    const double a = 0.5 * x, q = -a * a;
    // everything carries the exact factor 2^600 (|J_n| <= 1, so nothing overflows) so
    // that (x/2)^p / p! stays representable down to tiny x; it is removed at the end
    const double up = 0x1p600, down = 0x1p-600;
    double t = up;   // 2^600 a^p / p!
    for (int i = 1; i <= p; ++i) t *= a * k_inv_int[i];
    if (t < 1e-290) {   // x tiny: J_n = (x/2)^n / n! (1 + q / (n+1) + q^2 / (2 (n+1)(n+2))), error O(q^3)
        double tn = 1.0;
        for (int n = 0; n <= p; ++n) {
            if (n > 0) tn *= a * k_inv_int[n];
            out[n] = tn * (1.0 + q * k_inv_int[n + 1] * (1.0 + 0.5 * q * k_inv_int[n + 2]));
        }
        return;
    }
    double S1 = 1.0, S0 = 1.0, c1 = 1.0, c0 = 1.0;   // series of J_p and J_{p-1}
    for (int k = 1; k <= 40; ++k) {
        c1 *= q * k_inv_int[k] * k_inv_int[p + k];
        c0 *= q * k_inv_int[k] * k_inv_int[p - 1 + k];
        S1 += c1;
        S0 += c0;
        if (fabs(c1) <= 1e-17 * fabs(S1) && fabs(c0) <= 1e-17 * fabs(S0)) break;
    }
    const double ia = 1.0 / a;   // = 2 / x
    double jp = t * S1, jn = t * (p * ia) * S0;
    out[p] = jp * down;
    out[p - 1] = jn * down;
    for (int n = p - 1; n >= 1; --n) {
        const double jm = (n * ia) * jn - jp;
        out[n - 1] = jm * down;
        jp = jn;
        jn = jm;
    }
}

// Hankel functions H_n^(1)(x) for n = 0..p by forward recurrence from
// H_0 = J_0 + i Y_0 and H_1 = J_1 + i Y_1 (forward recurrence is stable for
// the dominant Y_n; the J_n part is negligible there).  x > 0.
__host__ __device__ inline void hankel_seq(double x, int p, cd* out) {
    out[0] = mk(j0(x), y0(x));
    if (p >= 1) out[1] = mk(j1(x), y1(x));
    for (int n = 1; n < p; ++n) {
        double f = 2.0 * n / x;
        out[n + 1] = mk(f * out[n].x - out[n - 1].x, f * out[n].y - out[n - 1].y);
    }
}

// ---------------------------------------------------------------------------
// Medium in constant memory and the reaction densities.
// ---------------------------------------------------------------------------
struct MediumDev {
    int nl;                       // L+1
    double yint[LFMM_MAXLAY];     // interface heights, decreasing
    double k[LFMM_MAXLAY];
    double eta[LFMM_MAXLAY];
    double kmax;
};

// Interface-referenced reaction density Sigma_c(lambda) of component
// (field layer ls with arrival a, source layer lt with departure b), 0 = up, 1 = down.
//
// This is the paper's Cases I-III (eqs. densityinsourcelayer, disity1, disity2)
// built on the generalized reflection recursions (eqs. Rellrecursionup,
// Rellrecursiondown) and the generalized transmission (eq. generaltransmission),
// multiplied by the factor i/(2 k_{l',y}) of the Sommerfeld representation,
// but with every wave referenced at the interface it last met instead of at
// y = 0: the transmission chain carries the layer phases e^{i k_m H_m}
// explicitly instead of the absolute factors e^{i (k_l - k_{l+1}) d_l}.  All
// factors then have modulus O(1) for Im k_y >= 0, which keeps the densities
// finite for evanescent lambda at any depth.  The full kernel is
//   G^{*star}_{ll'}(r, r') = (1/2pi) int Sigma(lambda) e^{i lambda (x-x')}
//                             e^{i k_{l,y} h_*(y)} e^{i k_{l',y} h_star(y')} d lambda
// with h_up(y) = y - y_l (field point above its bottom interface), h_down(y) =
// y_{l-1} - y, and at the source h_up(y') = y_{l'-1} - y', h_down(y') = y' - y_{l'}.
__host__ __device__ inline cd sigma_comp(const MediumDev& m, cd lam, int ls, int a, int lt, int b) {
    const int L = m.nl - 1;
    cd kyv[LFMM_MAXLAY], e[LFMM_MAXLAY];
    for (int q = 0; q <= L; ++q) {
        kyv[q] = ky_of(m.k[q], lam);
        if (q >= 1 && q <= L - 1) {
            double H = m.yint[q - 1] - m.yint[q];
            e[q] = cexpd(mk(-kyv[q].y * H, kyv[q].x * H));
        } else {
            e[q] = mk(0.0, 0.0);
        }
    }
    // local reflection R_{q,q+1} for q = 0..L-1
    cd Rl[LFMM_MAXLAY];
    for (int q = 0; q < L; ++q) {
        cd A = m.eta[q] * kyv[q], B = m.eta[q + 1] * kyv[q + 1];
        Rl[q] = cdiv(A - B, A + B);
    }
    // generalized reflections looking down (Rd[q] = R~_{q,q+1}) and up (Ru[q] = R~_{q,q-1})
    cd Rd[LFMM_MAXLAY], Ru[LFMM_MAXLAY];
    for (int q = 0; q <= L; ++q) { Rd[q] = mk(0.0, 0.0); Ru[q] = mk(0.0, 0.0); }
    for (int q = L - 1; q >= 0; --q) {
        if (q == L - 1) {
            Rd[q] = Rl[q];
        } else {
            cd t = Rd[q + 1] * (e[q + 1] * e[q + 1]);
            Rd[q] = cdiv(Rl[q] + t, mk(1.0, 0.0) + Rl[q] * t);
        }
    }
    for (int q = 1; q <= L; ++q) {
        cd r = -Rl[q - 1];
        if (q == 1) {
            Ru[q] = r;
        } else {
            cd t = Ru[q - 1] * (e[q - 1] * e[q - 1]);
            Ru[q] = cdiv(r + t, mk(1.0, 0.0) + r * t);
        }
    }
    const int lp = lt;
    cd Mden = mk(1.0, 0.0) - Ru[lp] * Rd[lp] * (e[lp] * e[lp]);
    cd base = cdiv(mk(0.0, 1.0), 2.0 * kyv[lp] * Mden);   // i / (2 k_{l',y} M)
    if (ls == lp) {
        if (a == 0 && b == 1) return base * Rd[lp];
        if (a == 1 && b == 0) return base * Ru[lp];
        return base * Rd[lp] * Ru[lp] * e[lp];
    }
    cd T = mk(1.0, 0.0);
    if (ls < lp) {   // field above the source: transmit upward through interfaces lp-1 .. ls
        for (int q = ls; q < lp; ++q) {
            cd A = m.eta[q] * kyv[q], B = m.eta[q + 1] * kyv[q + 1];
            cd Tup = cdiv(2.0 * B, A + B);                    // T_{q+1,q}
            cd den = mk(1.0, 0.0) - Rl[q] * Ru[q] * (e[q] * e[q]);
            T = cdiv(T * Tup, den);
        }
        for (int q = ls + 1; q < lp; ++q) T = T * e[q];
        cd v = base * T;
        if (a == 1) v = v * Ru[ls] * e[ls];
        if (b == 1) v = v * Rd[lp] * e[lp];
        return v;
    }
    // field below the source: transmit downward through interfaces lp .. ls-1
    for (int q = lp + 1; q <= ls; ++q) {
        cd A = m.eta[q - 1] * kyv[q - 1], B = m.eta[q] * kyv[q];
        cd Tdn = cdiv(2.0 * A, A + B);                         // T_{q-1,q}
        cd den = mk(1.0, 0.0) + Rl[q - 1] * Rd[q] * (e[q] * e[q]);   // 1 - R_{q,q-1} R~_{q,q+1} e^2
        T = cdiv(T * Tdn, den);
    }
    for (int q = lp + 1; q < ls; ++q) T = T * e[q];
    cd v = base * T;
    if (a == 0) v = v * Rd[ls] * e[ls];
    if (b == 0) v = v * Ru[lp] * e[lp];
    return v;
}

// e^{i k_y h} for real h (h may be slightly negative for box centres)
__host__ __device__ __forceinline__ cd eikh(cd kyv, double h) {
    return cexpd(mk(-kyv.y * h, kyv.x * h));
}

// ---- free-space entries of the Nystrom operators (Sec. 3.3) -------------------
// Single layer: (i/4) H_0(k r).  Combined field (opt-in second-kind form): the
// double layer n_e . grad_{c_e} (i/4) H_0(k |c_e - c_i|) = -(i/4) k H_1(k r)
// n_e . (c_e - c_i) / r plus -i kappa (i/4) H_0(k r) with the coupling kappa = k
// of the element's layer.  (dx, dy) = c_e - c_i != 0; (nx, ny) is n_e.
__host__ __device__ __forceinline__ cd free_kernel(double k, double dx, double dy, bool cf, double nx, double ny) {
    const double r = hypot(dx, dy), z = k * r;
    const cd g = mk(-0.25 * y0(z), 0.25 * j0(z));   // (i/4)(J_0 + i Y_0)
    if (!cf) return g;
    const double c = -k * (nx * dx + ny * dy) / r;
    return mk(c * -0.25 * y1(z) + k * g.y, c * 0.25 * j1(z) - k * g.x);
}
// Diagonal entry: the single-layer self term I^s (eq. ApproximateComputation) or,
// for the combined field, 1/2 (the exterior jump of the double layer; the double
// layer of a straight element on its own centre vanishes) - i k I^s.
__host__ __device__ __forceinline__ cd self_entry(double k, double w, bool cf) {
    const double eg = 0.57721566490153286060651209008240243;
    const cd is = mk(-(eg + log(k * w / 4.0) - 1.0) / (2.0 * M_PI) * w, 0.25 * w);
    if (!cf) return is;
    return mk(0.5 + k * is.y, -k * is.x);
}
