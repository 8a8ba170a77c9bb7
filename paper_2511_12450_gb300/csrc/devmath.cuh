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
// fused a += b * c
__host__ __device__ __forceinline__ void cfma(cd& a, cd b, cd c) {
    a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
    a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}
__device__ __forceinline__ cd cexpd(cd z) {
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
__device__ __forceinline__ cd w_of(cd kyv, cd lam, double k) {
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

// Hankel functions H_n^(1)(x) for n = 0..p by forward recurrence from
// H_0 = J_0 + i Y_0 and H_1 = J_1 + i Y_1 (forward recurrence is stable for
// the dominant Y_n; the J_n part is negligible there).  x > 0.
__device__ inline void hankel_seq(double x, int p, cd* out) {
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
__device__ inline cd sigma_comp(const MediumDev& m, cd lam, int ls, int a, int lt, int b) {
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
__device__ __forceinline__ cd eikh(cd kyv, double h) {
    return cexpd(mk(-kyv.y * h, kyv.x * h));
}
