// mixed.cu -- the precision form of the operator: on the levels whose order is
// at most 1.5 p, the whole far field -- P2M, M2M, the multipole-to-local
// translations (free space, Graf's addition theorem, and the reaction
// components' moment tables of eq. generalintegral), L2L and L2P -- in FP32;
// the coarser wide-band levels, the stored near field with its singular and
// Sommerfeld entries, and every sum into the FP64 output stay FP64.
//
// FP32 has 8 exponent bits; the expansions span far more.  At the fine levels
// the multipole coefficients decay like (k rho / 2)^n / n! and the Hankel
// translation entries H_{m-n}(k R) grow like (|m-n| - 1)! (2 / k R)^{|m-n|}
// (J_20(0.2) ~ 1e-38 and H_40(0.6) ~ 1e66 at the C2 leaf level).  Every
// expansion of a (layer, level) is therefore carried scaled,
//     M~_n = M_n / s^|n|,     L~_n = L_n s^|n|,
// and the translation operators accordingly,
//     free:      L~_n = sum_m [s^(|n| + |m|) T_{m-n}] M~_m,
//     reaction:  beta~_m = sum_n [s_T^|m| s_S^|n| I_{mn}] alpha~_n,
// with s <= 1 chosen per (layer, level) on the host so that the scaled basis
// values and translation entries stay well inside the FP32 range.  The scaled
// operators are stored as dense FP32 matrices (column-major): free-space M2L per
// (layer, level, offset), reaction M2L per moment table, M2M / L2L per source of
// every destination of the FP32 passes.  At the first FP32 level the FP32
// multipoles are converted to FP64 for the coarser levels, and the FP64
// parent-to-child locals are added into the FP32 ones.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dfloat.cuh"
#include "geometry.h"

namespace lfmm {

struct cf {
    float x, y;
};
__device__ __forceinline__ cf mkf(float a, float b) { cf r; r.x = a; r.y = b; return r; }
__device__ __forceinline__ void cfmaf(cf& a, cf b, cf c) {
    a.x = fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x));
    a.y = fmaf(b.x, c.y, fmaf(b.y, c.x, a.y));
}
__device__ __forceinline__ cf addf(cf a, cf b) { return mkf(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cf mulf(cf a, cf b) { return mkf(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)); }
// point t of a P2M / L2P group: its entry (relative index) and point index
__device__ __forceinline__ void group_point32(const ExpEntry* __restrict__ ent, int e0, int e1, int t, int* er, int* j) {
    int e = e0, base = 0;
    while (e + 1 < e1 && t >= base + (ent[e].end - ent[e].beg)) { base += ent[e].end - ent[e].beg; ++e; }
    *er = e - e0;
    *j = ent[e].beg + (t - base);
}

struct MixedState {
    int cols = 0;                       // right-hand-side columns the FP32 buffers hold
    cf *M = nullptr, *L = nullptr;      // [cols][ncoef]   scaled multipoles / locals
    cf *Mp = nullptr, *Lp = nullptr;    // [cols][nslotcoef]
    cf *part = nullptr;                 // M2L partial sums [cols][parts][3][XT_W]
    double *ispow = nullptr;            // [ncoef]      s^-|n| per coefficient
    double *ispow_slot = nullptr;       // [nslotcoef]
    cf *ftab = nullptr;                 // scaled dense free-space tables
    int64_t *ftab_off = nullptr;        // per table id
    cf *rtab = nullptr;                 // scaled dense reaction tables (offsets as ReactKey::off)
    std::vector<double> scale;          // [layer * nlev + level]
    double* d_scale = nullptr;          // device copy
    int lm = 0;                         // first FP32 level
    cf* wtab = nullptr;                 // dense scaled M2M / L2L tables of the FP32 passes
    int64_t* wtab_off = nullptr;        // per XSrc (-1 outside the FP32 passes)
    int* d_xd_layer = nullptr;          // layer per XDst
    // cell families: base table per ((child level 2 + down) nl + layer), and the records
    // k_xtab32 builds them from
    int64_t* qoff = nullptr;
    XDst* q_bd = nullptr;
    XSrc* q_bs = nullptr;
    int* q_blay = nullptr;
    int64_t* q_bwoff = nullptr;
    size_t smem_p2m = 0, smem_l2p = 0;
    size_t bytes = 0;
    // block right-hand-side M2L on the tensor cores (m2l_tc.cuh)
    int* tc_boxes = nullptr;            // boxes of the FP32 levels, one CTA each
    int n_tc_boxes = 0;
    int* tc_ent_ptr = nullptr;          // list-entry range per box
    int tc_p = 0;                       // largest expansion order of the FP32 levels (the coarsest)
    int* tc_err = nullptr;              // set when an mbarrier wait of k_m2l32_tc gave up
    int* tc_err_host = nullptr;         // pinned copy, read at the next call
    // the coarse (wide-band) levels' M2L in double-float (levels l0 .. lm - 1)
    dfc* ftab_df = nullptr;             // [2][m2lf_len]: scaled and unscaled Toeplitz vectors (offsets d_m2lf_off)
    dfc* rtab_df = nullptr;             // scaled reaction tables of those levels (offsets as ReactKey::off)
    float* rtab_rsc = nullptr;          // their row factors 2^e_m (at ReactKey::off + row)
    dfc *Mdf = nullptr, *Mudf = nullptr, *Mpdf = nullptr;   // [cols][ncd] scaled / unscaled, [cols][nsd]
    int* df_emax = nullptr;             // [cols] exponent bound of each column's coarse multipoles
    int64_t df_c0 = 0, df_ncd = 0, df_s0 = 0, df_nsd = 0;  // coefficient ranges of those levels
    int df_cols = 0;
    bool df_ok = false;                 // the coarse levels' M2L runs in double-float
    double df_range[3] = {0, 0, 0};     // log10: largest free-space, reaction table component; scaled basis
};

// ---------------------------------------------------------------------------
// Choice of the scale s for one (layer, level).
// log10 of the largest scaled translation entry: max_{j <= 2p} s^j |Y_j(k 2w)|
// (2w is the smallest centre distance of an M2L pair; |H_j| ~ |Y_j| where it is
// large), by the forward recurrence of Y_j with running rescaling.
static double log10_max_scaled_y(double x, int jmax, double s) {
    double y0 = std::cyl_neumann(0.0, x), y1 = std::cyl_neumann(1.0, x);
    double lsc = 0.0;   // log10 of the factor divided out of (y0, y1)
    double best = std::log10(std::max(std::fabs(y0), 1e-300));
    best = std::max(best, std::log10(std::max(std::fabs(y1), 1e-300)) + std::log10(s));
    for (int j = 1; j < jmax; ++j) {
        double y2 = (2.0 * j / x) * y1 - y0;
        y0 = y1;
        y1 = y2;
        double a = std::fabs(y1);
        if (a > 1e200) { y0 *= 1e-200; y1 *= 1e-200; lsc += 200.0; a = std::fabs(y1); }
        best = std::max(best, std::log10(std::max(a, 1e-300)) + lsc + (j + 1) * std::log10(s));
    }
    return best;
}
// log10 of the envelope of |J_n(x)|: 0 while n <= x, else the leading term of the
// power series, (x/2)^n / n! (the envelope avoids the zeros of J_n).
static double log10_env_j(double x, int n) {
    const double lead = n * std::log10(0.5 * x) - std::lgamma(n + 1.0) / std::log(10.0);
    return std::min(0.0, lead);
}
// The scale keeps three magnitudes inside the FP32 range at once: the largest
// scaled multipole basis value max_n |J_n(x)| / s^n, the smallest one
// |J_p(x)| / s^p (x = k w / sqrt(2), the farthest point of the box), and the
// largest scaled translation entry.  s is a power of two in (0, 1]; the chosen
// one minimises the largest of the three log-magnitudes.
// big_m_out (optional) receives log10 of the largest scaled basis value at the chosen s.
static double choose_scale(double k, double w, int p, double* big_m_out = nullptr) {
    const double x = k * w / std::sqrt(2.0);
    double best_s = 1.0, best_v = 1e300, best_m = 0.0;
    for (int j = 0; j <= 80; ++j) {
        const double s = std::ldexp(1.0, -j), ls = std::log10(s);
        double big_m = -1e300;
        for (int n = 0; n <= p; ++n) big_m = std::max(big_m, log10_env_j(x, n) - n * ls);
        const double small_m = log10_env_j(x, p) - p * ls;
        const double big_t = log10_max_scaled_y(2.0 * k * w, 2 * p, s);
        const double v = std::max(std::max(big_m, big_t), -small_m);
        if (v < best_v) { best_v = v; best_s = s; best_m = big_m; }
    }
    if (big_m_out) *big_m_out = best_m;
    return best_s;
}

// ---------------------------------------------------------------------------
// Table and coefficient conversions.
__global__ void k_free32_tables(const cd* __restrict__ m2lf, const int64_t* __restrict__ m2lf_off,
                                const int* __restrict__ tab_p, const double* __restrict__ tab_s,
                                const int64_t* __restrict__ off32, cf* __restrict__ out) {
    const int id = blockIdx.x;
    const int p = tab_p[id], nco = 2 * p + 1;
    const double s = tab_s[id];
    const cd* base = m2lf + m2lf_off[id];
    for (int e = threadIdx.x; e < nco * nco; e += blockDim.x) {
        const int mi = e / nco, ni = e - mi * nco;   // column-major: (n_out, m_in) at m_in nco + n_out
        const int n = ni - p, m = mi - p;
        const double f = pow(s, (double)(abs(n) + abs(m)));
        const cd v = base[mi - ni + 2 * p];          // T_{m-n}
        out[off32[id] + e] = mkf((float)(f * v.x), (float)(f * v.y));
    }
}
__global__ void k_react32_tables(const cd* __restrict__ m2lr, const ReactKey* __restrict__ keys,
                                 const double* __restrict__ key_ss, const double* __restrict__ key_st,
                                 cf* __restrict__ out) {
    const ReactKey K = keys[blockIdx.x];
    const int ncT = 2 * K.pT + 1, ncS = 2 * K.pS + 1;
    const double ss = key_ss[blockIdx.x], st = key_st[blockIdx.x];
    for (int e = threadIdx.x; e < ncT * ncS; e += blockDim.x) {
        const int ni = e / ncT, mi = e - ni * ncT;   // column-major: (m_out, n_in) at n_in ncT + m_out
        const double f = pow(st, (double)abs(mi - K.pT)) * pow(ss, (double)abs(ni - K.pS));
        const cd v = m2lr[K.off + e];
        out[K.off + e] = mkf((float)(f * v.x), (float)(f * v.y));
    }
}

// ---------------------------------------------------------------------------
// M2L in FP32 on the scaled expansions: the same work items, entry descriptors,
// lane/slice split, index flips and partial-sum reduction as the FP64 kernel,
// with dense tables for the free-space part too.
#define M2L_STAGE32 64
// v or -v by flipping the sign bits with integer instructions (a conditional
// negation otherwise takes a floating-point instruction in the inner loop)
__device__ __forceinline__ cf csignf(cf v, int neg) {
    const unsigned msk = (unsigned)(neg & 1) << 31;
    return mkf(__uint_as_float(__float_as_uint(v.x) ^ msk), __uint_as_float(__float_as_uint(v.y) ^ msk));
}
__global__ void __launch_bounds__(128) k_m2l32(const M2LItem* __restrict__ items, const M2LEnt* __restrict__ ents,
                        const int* __restrict__ box_level, const int* __restrict__ p_level,
                        const int64_t* __restrict__ coef_off, const int* __restrict__ slot_of,
                        const int64_t* __restrict__ slot_coef, const cf* __restrict__ ftab,
                        const int64_t* __restrict__ ftab_off, const cf* __restrict__ rtab, int nrhs, int64_t ncoef,
                        int64_t nslotcoef, int nparts, const cf* __restrict__ Min, const cf* __restrict__ Mp,
                        cf* __restrict__ Lout, cf* __restrict__ Lp, cf* __restrict__ part) {
    __shared__ cf red[3 * 128];
    __shared__ M2LEnt se[M2L_STAGE32];
    const M2LItem it = items[blockIdx.x];
    const int T = it.box;
    const int p = p_level[box_level[T]];
    const int nco = 2 * p + 1;
    const int W = it.w, NS = 128 / W;
    const int lane = threadIdx.x % W, sl = threadIdx.x / W;
    const int idx = it.chunk * W + lane;
    const bool live = sl < NS && idx < nco;
    const int nn = idx - p;
    for (int col = 0; col < nrhs; ++col) {
        const cf* Mc = Min + (int64_t)col * ncoef;
        const cf* Mpc = Mp + (int64_t)col * nslotcoef;
        cf acc0 = mkf(0, 0), acc1 = mkf(0, 0), acc2 = mkf(0, 0);
        for (int eb = it.e0; eb < it.e1; eb += M2L_STAGE32) {
            const int cnt = min(M2L_STAGE32, it.e1 - eb);
            __syncthreads();
            if (threadIdx.x < cnt) se[threadIdx.x] = ents[eb + threadIdx.x];
            __syncthreads();
            if (!live) continue;
            for (int q = 0; q < cnt; ++q) {
                const M2LEnt E = se[q];
                if (!(E.flags & M2L_REACT)) {
                    const cf* src = Mc + E.src;
                    const cf* tb = ftab + ftab_off[E.tab] + idx;   // (n_out, m_in) at m_in nco + n_out
                    for (int mi = sl; mi < nco; mi += NS) cfmaf(acc0, src[mi], tb[mi * nco]);
                } else {
                    const cf* src = ((E.flags & M2L_SRC_SLOT) ? Mpc : Mc) + E.src;
                    const bool bdown = (E.flags & M2L_B_DOWN) != 0;
                    const int mrow = bdown ? nn : -nn;
                    // column of row mrow; a mirrored table is read at (-mrow, -n)
                    const bool flip = (E.flags & M2L_FLIP) != 0;
                    const cf* col_m = rtab + E.tab + (flip ? (p - mrow) + (int64_t)2 * p * nco : (mrow + p));
                    const int64_t cs = flip ? -(int64_t)nco : (int64_t)nco;
                    cf bsum = mkf(0, 0);
                    if (E.flags & M2L_A_DOWN) {
                        for (int mi = sl; mi < nco; mi += NS) cfmaf(bsum, col_m[mi * cs], src[mi]);
                    } else {
                        for (int mi = sl; mi < nco; mi += NS) cfmaf(bsum, col_m[mi * cs], csignf(src[2 * p - mi], mi - p));
                    }
                    bsum = csignf(bsum, (!bdown) & mrow);
                    const int dst = (E.flags >> M2L_DST_SHIFT) & 3;
                    if (dst == 0) acc0 = addf(acc0, bsum);
                    else if (dst == 1) acc1 = addf(acc1, bsum);
                    else acc2 = addf(acc2, bsum);
                }
            }
        }
        if (sl < NS) {
            red[(0 * NS + sl) * W + lane] = acc0;
            red[(1 * NS + sl) * W + lane] = acc1;
            red[(2 * NS + sl) * W + lane] = acc2;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * W; i += blockDim.x) {
            const int k = i / W, ln = i - k * W, ix = it.chunk * W + ln;
            if (ix >= nco) continue;
            cf t = red[(k * NS) * W + ln];
            for (int q = 1; q < NS; ++q) t = addf(t, red[(k * NS + q) * W + ln]);
            if (it.part >= 0) {   // split items are always XT_W lanes wide
                part[(((int64_t)col * nparts + it.part) * 3 + k) * XT_W + ln] = t;
            } else {
                const int ts = (k == 0) ? -1 : slot_of[2 * T + k - 1];
                if (k == 0) Lout[(int64_t)col * ncoef + coef_off[T] + ix] = t;
                else if (ts >= 0) Lp[(int64_t)col * nslotcoef + slot_coef[ts] + ix] = t;
            }
        }
        __syncthreads();
    }
}
__global__ void __launch_bounds__(64) k_m2l32_reduce(const M2LReduce* __restrict__ reds,
                        const int* __restrict__ box_level, const int* __restrict__ p_level,
                        const int64_t* __restrict__ coef_off, const int* __restrict__ slot_of,
                        const int64_t* __restrict__ slot_coef, int nrhs, int64_t ncoef, int64_t nslotcoef, int nparts,
                        const cf* __restrict__ part, cf* __restrict__ Lout, cf* __restrict__ Lp) {
    const M2LReduce r = reds[blockIdx.x];
    const int p = p_level[box_level[r.box]];
    const int lane = threadIdx.x % XT_W, k = threadIdx.x / XT_W;
    const int idx = r.chunk * XT_W + lane;
    if (k >= 3 || idx >= 2 * p + 1) return;
    const int ts = (k == 0) ? -1 : slot_of[2 * r.box + k - 1];
    if (k > 0 && ts < 0) return;
    for (int col = 0; col < nrhs; ++col) {
        cf t = mkf(0, 0);
        for (int q = 0; q < r.nparts; ++q) t = addf(t, part[(((int64_t)col * nparts + r.part0 + q) * 3 + k) * XT_W + lane]);
        if (k == 0) Lout[(int64_t)col * ncoef + coef_off[r.box] + idx] = t;
        else Lp[(int64_t)col * nslotcoef + slot_coef[ts] + idx] = t;
    }
}

#include "m2l_tc.cuh"

// ---------------------------------------------------------------------------
// Scaled Bessel values in FP32: out[n] = J_n(x) / s^n, n = 0..p, from the power
// series J_n(x) = (x/2)^n / n! sum_k (-x^2/4)^k / (k! (n+1)...(n+k)) (A&S 9.1.10),
// i.e. t_n S_n with t_n = a^n / n!, a = x / (2 s).  Used at the leaves of the
// levels that run in FP32, where x = k rho stays below the order p; no overflow
// (t_n and the series terms are bounded there by the choice of s), no
// normalisation step.
__device__ __forceinline__ void bessel_j_scaled_f(float x, float s, int p, float* out) {
    const float a = x / (2.0f * s);
    const float q = -0.25f * x * x;
    float t = 1.0f;
    for (int n = 0; n <= p; ++n) {
        if (n > 0) t *= a / (float)n;
        float c = 1.0f, S = 1.0f;
        for (int k = 1; k <= 40; ++k) {
            c *= q / (float)(k * (n + k));
            S += c;
            if (fabsf(c) <= 1e-9f * fabsf(S)) break;
        }
        out[n] = t * S;
    }
}

// P2M in FP32 at the leaves (cell centres and straddling leaves' reaction centres):
// M~_n = sum_j q_j J_n(k rho_j) e^{-i n theta_j} / s^|n|.  Same grouping and
// phases as the FP64 kernel.  Combined field (normals given): the scaled dipole +
// charge basis E_n / s^|n| = k [ (conj(nu) u~_{n-1} s^{|n-1|-|n|} - nu u~_{n+1}
// s^{|n+1|-|n|}) / 2 - i u~_n ] with u~_m = u_m / s^|m|, stored for every n.
__global__ void __launch_bounds__(128) k_p2m32(const ExpGroup* __restrict__ groups, const ExpEntry* __restrict__ ent,
                        MediumDev m, const double* __restrict__ sc, int lev, int nlev,
                        const double* __restrict__ px, const double* __restrict__ py, const double* __restrict__ pw,
                        const double* __restrict__ nx, const double* __restrict__ ny,
                        const cd* __restrict__ phi, int64_t n, int nrhs, int64_t stride, cf* __restrict__ M) {
    extern __shared__ cf su32[];   // [npts][rs] u, then [npts] q, then [nent + 1] offsets
    const ExpGroup G = groups[blockIdx.x];
    const int p = ent[G.e0].p, nco = 2 * p + 1;
    const bool cfm = nx != nullptr;
    // rows: u~_0..u~_p (single layer; negative orders by symmetry in phase 2), or the
    // combined-field basis for n = -p..p in a row of 2p + 3 (room for u~_{-p-1..p+1})
    const int pb = cfm ? p + 1 : p, rs = cfm ? 2 * p + 3 : p + 1, o0 = cfm ? p + 1 : 0;
    const int ne = G.e1 - G.e0;
    cf* sq = su32 + (size_t)G.npts * rs;
    int* soff = (int*)(sq + G.npts);
    if (threadIdx.x == 0) {
        int o = 0;
        for (int e = 0; e < ne; ++e) { soff[e] = o; o += ent[G.e0 + e].end - ent[G.e0 + e].beg; }
        soff[ne] = o;
    }
    for (int t = threadIdx.x; t < G.npts; t += blockDim.x) {
        int er, j;
        group_point32(ent, G.e0, G.e1, t, &er, &j);
        const ExpEntry& E = ent[G.e0 + er];
        const double dx = px[j] - E.cx, dy = py[j] - E.cy;
        const double rho = hypot(dx, dy);
        cf* u = su32 + (size_t)t * rs + o0;
        // u_n = J~_n z^n, z = e^{-i theta}, upward from z^0 = 1 so the low orders carry
        // the least rounding
        const float x = (float)(m.k[E.lay] * rho), sf = (float)sc[E.lay * nlev + lev];
        const float a = x / (2.0f * sf), q = -0.25f * x * x;
        const cf z = (rho > 0.0) ? mkf((float)(dx / rho), (float)(-dy / rho)) : mkf(1.0f, 0.0f);
        cf zn = mkf(1.0f, 0.0f);
        float tn = 1.0f;
        for (int k2 = 0; k2 <= pb; ++k2) {
            if (k2 > 0) { tn *= a / (float)k2; zn = mulf(zn, z); }
            float c = 1.0f, S = 1.0f;
            for (int k = 1; k <= 40; ++k) {
                c *= q / (float)(k * (k2 + k));
                S += c;
                if (fabsf(c) <= 1e-9f * fabsf(S)) break;
            }
            const float jv = tn * S;
            u[k2] = mkf(jv * zn.x, jv * zn.y);
        }
        if (cfm) {
            for (int k2 = 1; k2 <= pb; ++k2) {   // u~_{-m} = (-1)^m conj(u~_m)
                const cf v = u[k2];
                u[-k2] = (k2 & 1) ? mkf(-v.x, v.y) : mkf(v.x, -v.y);
            }
            // E~_n into row slot n + p from u~_{n-1}, u~_n, u~_{n+1} (row slots n+p .. n+p+2);
            // ascending n overwrites only u~_{n-1}
            cf* row = u - o0;
            const float k = (float)m.k[E.lay], isf = 1.0f / sf;
            const cf nu = mkf((float)nx[j], (float)ny[j]);
            for (int s2 = 0; s2 < nco; ++s2) {
                const int nn = s2 - p;
                const float fm = (nn >= 1) ? isf : sf, fp = (nn <= -1) ? isf : sf;
                const cf um = row[s2], u0 = row[s2 + 1], up = row[s2 + 2];
                // conj(nu) um fm - nu up fp
                const float dx2 = fm * (nu.x * um.x + nu.y * um.y) - fp * (nu.x * up.x - nu.y * up.y);
                const float dy2 = fm * (nu.x * um.y - nu.y * um.x) - fp * (nu.x * up.y + nu.y * up.x);
                row[s2] = mkf(k * (0.5f * dx2 + u0.y), k * (0.5f * dy2 - u0.x));
            }
        }
    }
    for (int col = 0; col < nrhs; ++col) {
        __syncthreads();
        for (int t = threadIdx.x; t < G.npts; t += blockDim.x) {
            int er, j;
            group_point32(ent, G.e0, G.e1, t, &er, &j);
            const cd qv = pw[j] * phi[(int64_t)col * n + j];
            sq[t] = mkf((float)qv.x, (float)qv.y);
        }
        __syncthreads();
        for (int task = threadIdx.x; task < ne * nco; task += blockDim.x) {
            const int er = task / nco, idx = task - er * nco;
            const int nn = idx - p, an = nn < 0 ? -nn : nn;
            cf acc = mkf(0, 0);
            if (cfm) {
                for (int t = soff[er]; t < soff[er + 1]; ++t) cfmaf(acc, sq[t], su32[(size_t)t * rs + idx]);
            } else {
                for (int t = soff[er]; t < soff[er + 1]; ++t) {
                    cf v = su32[(size_t)t * rs + an];
                    if (nn < 0) { v.y = -v.y; if (an & 1) { v.x = -v.x; v.y = -v.y; } }
                    cfmaf(acc, sq[t], v);
                }
            }
            M[(int64_t)col * stride + ent[G.e0 + er].off + idx] = acc;
        }
    }
}

// L2P in FP32 at the leaves: y_j += sum_n L~_n J_n(k rho_j) e^{i n theta_j} / s^|n|
// (the result is added to the FP64 output).
__global__ void __launch_bounds__(128) k_l2p32(const ExpGroup* __restrict__ groups, const ExpEntry* __restrict__ ent,
                        MediumDev m, const double* __restrict__ sc, int lev, int nlev,
                        const double* __restrict__ px, const double* __restrict__ py, int64_t n, int nrhs,
                        int64_t stride, const cf* __restrict__ L, cd* __restrict__ y) {
    extern __shared__ float sj32[];   // [npts][p+1] J~, then [nent][2p+1] coefficients
    const ExpGroup G = groups[blockIdx.x];
    const int p = ent[G.e0].p, np1 = p + 1, nco = 2 * p + 1;
    const int ne = G.e1 - G.e0;
    cf* sL = (cf*)(sj32 + (((size_t)G.npts * np1 + 1) & ~(size_t)1));
    for (int col = 0; col < nrhs; ++col) {
        __syncthreads();
        for (int i = threadIdx.x; i < ne * nco; i += blockDim.x) {
            const int er = i / nco, idx = i - er * nco;
            sL[i] = L[(int64_t)col * stride + ent[G.e0 + er].off + idx];
        }
        __syncthreads();
        for (int t = threadIdx.x; t < G.npts; t += blockDim.x) {
            int er, j;
            group_point32(ent, G.e0, G.e1, t, &er, &j);
            const ExpEntry& E = ent[G.e0 + er];
            const double dx = px[j] - E.cx, dy = py[j] - E.cy;
            const double rho = hypot(dx, dy);
            float* J = sj32 + (size_t)t * np1;
            if (col == 0) bessel_j_scaled_f((float)(m.k[E.lay] * rho), (float)sc[E.lay * nlev + lev], p, J);
            const cf z = (rho > 0.0) ? mkf((float)(dx / rho), (float)(dy / rho)) : mkf(1.0f, 0.0f);
            const cf* Le = sL + er * nco;
            cf acc = mkf(Le[p].x * J[0], Le[p].y * J[0]);
            cf zz = mkf(1.0f, 0.0f);
            for (int k2 = 1; k2 <= p; ++k2) {
                zz = mulf(zz, z);
                const float jt = J[k2];
                const cf a1 = Le[p + k2], a2 = Le[p - k2];
                const float js = (k2 & 1) ? -jt : jt;
                cfmaf(acc, mkf(jt * a1.x, jt * a1.y), zz);
                cfmaf(acc, mkf(js * a2.x, js * a2.y), mkf(zz.x, -zz.y));
            }
            cd* yo = y + (int64_t)col * n + j;
            *yo = *yo + mk((double)acc.x, (double)acc.y);
        }
    }
}

// M2M / L2L in FP32 on scaled expansions, one launch per level and pass over the same
// two kinds of work item as the FP64 pass (k_translate): cell families in the quadrant
// form, with the base table W_B of the family's layer, and reaction-centre destinations,
//   out_n (= or +=) sum_j sum_m src_j[m] W_j[m][n].
// The tables are dense (column-major, (n, m) at m ncD + n) with the scale factors folded
// in.  The factors depend on |m| and |n| only, so the quadrant phases factor out of the
// scaled tables as they do of the vectors.
struct XPass32 {
    const XDst* dsts;
    const XSrc* srcs;
    const int64_t* wtab_off;   // per XSrc
    const cf* wtab;
    const QuadX* qx;
    const int64_t* qoff;       // base table of each layer (this level and pass)
    int nq, nd, nch, w, fch, fr, pS, pD, down, accumulate;
    int64_t ncoef, nslotcoef;
    cf *X, *Xp;
};
__device__ __forceinline__ cf subf(cf a, cf b) { return mkf(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cf mul_if(cf v) { return mkf(-v.y, v.x); }   // i v

__device__ __forceinline__ void translate32_dst(int di, int chunk, const XPass32& P, int col0, int col1, cf* red) {
    const XDst d = P.dsts[di];
    const int w = P.w, ns = 128 / w;
    const int lane = threadIdx.x % w, sl = threadIdx.x / w;
    const int idx = chunk * w + lane;
    const int ncD = 2 * d.p + 1;
    const bool live = sl < ns && idx < ncD;
    for (int col = col0; col < col1; ++col) {
        cf a = mkf(0, 0);
        if (live) {
            for (int j = d.src_begin; j < d.src_end; ++j) {
                const XSrc sr = P.srcs[j];
                const cf* src = (sr.in_slots ? P.Xp + (int64_t)col * P.nslotcoef : P.X + (int64_t)col * P.ncoef) + sr.off;
                const cf* W = P.wtab + P.wtab_off[j] + idx;
                const int ncS = 2 * sr.p + 1;
                for (int mi = sl; mi < ncS; mi += ns) cfmaf(a, src[mi], W[mi * ncD]);
            }
        }
        if (sl < ns) red[sl * w + lane] = a;
        __syncthreads();
        if (sl == 0 && idx < ncD) {
            cf t = red[lane];
            for (int q = 1; q < ns; ++q) t = addf(t, red[q * w + lane]);
            cf* dst = (d.in_slots ? P.Xp + (int64_t)col * P.nslotcoef : P.X + (int64_t)col * P.ncoef) + d.off + idx;
            if (P.accumulate) *dst = addf(*dst, t);
            else *dst = t;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ cf shfl_xor_cf(cf v, int m) {
    return mkf(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// the FP32 family passes: the warp design of fam_up / fam_dn (two rounds per lane at
// once) with the base table W_B (W_B[m][n] at m ncD + n) in place of the base vector
__device__ __forceinline__ void fam_up32(int fam, int chunk, const XPass32& P, int col0, int col1, cf* S) {
    const QuadX f = P.qx[fam];
    const int lane = threadIdx.x & 31, s = lane & 3;
    const int ncS = 2 * P.pS + 1, ncD = 2 * P.pD + 1;
    const cf* W = P.wtab + P.qoff[f.lay];
    const cf z = mkf(0, 0);
    for (int col = col0; col < col1; ++col) {
        const cf* Xc = P.X + (int64_t)col * P.ncoef;
        __syncwarp();
        for (int mi = lane; mi < ncS; mi += 32) {
            // om_q = 1, -i, -1, i for the quadrants 3, 2, 0, 1
            const cf m0 = f.ch[0] >= 0 ? Xc[f.ch[0] + mi] : z, m1 = f.ch[1] >= 0 ? Xc[f.ch[1] + mi] : z;
            const cf m2 = f.ch[2] >= 0 ? Xc[f.ch[2] + mi] : z, m3 = f.ch[3] >= 0 ? Xc[f.ch[3] + mi] : z;
            const cf u = addf(m3, m0), v = addf(m2, m1), x = subf(m3, m0), iy = mul_if(subf(m2, m1));
            S[mi] = addf(u, v);
            S[ncS + mi] = subf(x, iy);
            S[2 * ncS + mi] = subf(u, v);
            S[3 * ncS + mi] = addf(x, iy);
        }
        __syncwarp();
        const cf* Ss = S + s * ncS;
        for (int k = 0; k < P.fr; k += 2) {
            const int ni = (((chunk * P.fr + k) << 5) + lane) >> 2;
            const bool two = k + 1 < P.fr;
            cf a = z, a2 = z;
            if (ni < ncD) {
                const int mi0 = (ni - P.pD + P.pS - s) & 3;
                if (two) {
                    const int ni2 = min(ni + 8, ncD - 1);   // past the last output: not stored (as fam_up)
                    for (int mi = mi0; mi < ncS; mi += 4) {
                        const cf sv = Ss[mi];
                        cfmaf(a, sv, W[mi * ncD + ni]);
                        cfmaf(a2, sv, W[mi * ncD + ni2]);
                    }
                } else {
                    for (int mi = mi0; mi < ncS; mi += 4) cfmaf(a, Ss[mi], W[mi * ncD + ni]);
                }
            }
            a = addf(a, shfl_xor_cf(a, 1));
            a = addf(a, shfl_xor_cf(a, 2));
            if (s == 0 && ni < ncD) P.X[(int64_t)col * P.ncoef + f.par + ni] = a;
            if (two) {
                a2 = addf(a2, shfl_xor_cf(a2, 1));
                a2 = addf(a2, shfl_xor_cf(a2, 2));
                if (s == 0 && ni + 8 < ncD) P.X[(int64_t)col * P.ncoef + f.par + ni + 8] = a2;
            }
        }
    }
}

// the lane transform of fam_dn (quad_lane_transform) in FP32
__device__ __forceinline__ cf quad_lane_transform32(cf a, int s) {
    const cf o2 = shfl_xor_cf(a, 2);
    const cf b = (s < 2) ? addf(a, o2) : subf(o2, a);
    const cf o1 = shfl_xor_cf(b, 1);
    return (s == 0) ? addf(b, o1) : (s == 1) ? subf(o1, b) : (s == 2) ? addf(b, mul_if(o1)) : subf(o1, mul_if(b));
}

__device__ __forceinline__ void fam_dn32(int fam, int chunk, const XPass32& P, int col0, int col1) {
    const QuadX f = P.qx[fam];
    const int lane = threadIdx.x & 31, s = lane & 3;
    const int ncS = 2 * P.pS + 1, ncD = 2 * P.pD + 1;
    const int q = (0x1203 >> (4 * s)) & 15;   // the child lane s holds after the transform
    const int64_t chq = ((f.dn_skip >> q) & 1) ? -1 : P.qx[fam].ch[q];
    const cf* W = P.wtab + P.qoff[f.lay];
    const cf z = mkf(0, 0);
    for (int col = col0; col < col1; ++col) {
        const cf* src = P.X + (int64_t)col * P.ncoef + f.par;
        cf* Xc = P.X + (int64_t)col * P.ncoef + chq;
        for (int k = 0; k < P.fr; k += 2) {
            const int ni = (((chunk * P.fr + k) << 5) + lane) >> 2;
            const bool two = k + 1 < P.fr;
            cf a = z, a2 = z;
            if (ni < ncD) {
                const int mi0 = (ni - P.pD + P.pS + s) & 3;
                if (two) {
                    const int ni2 = min(ni + 8, ncD - 1);
                    for (int mi = mi0; mi < ncS; mi += 4) {
                        const cf sv = src[mi];
                        cfmaf(a, sv, W[mi * ncD + ni]);
                        cfmaf(a2, sv, W[mi * ncD + ni2]);
                    }
                } else {
                    for (int mi = mi0; mi < ncS; mi += 4) cfmaf(a, src[mi], W[mi * ncD + ni]);
                }
            }
            const cf out = quad_lane_transform32(a, s);
            if (ni < ncD && chq >= 0) Xc[ni] = P.accumulate ? addf(Xc[ni], out) : out;
            if (two) {
                const cf out2 = quad_lane_transform32(a2, s);
                if (ni + 8 < ncD && chq >= 0) Xc[ni + 8] = P.accumulate ? addf(Xc[ni + 8], out2) : out2;
            }
        }
    }
}

// GROUPS: the columns split over blockIdx.z in groups of four (col_groups); otherwise every
// CTA walks all columns (the single-column form keeps its registers)
template <bool GROUPS>
__global__ void __launch_bounds__(128) k_translate32(const XPass32 P, int nrhs) {
    extern __shared__ cf xsm32[];
    const int col0 = GROUPS ? blockIdx.z * 4 : 0, col1 = GROUPS ? min(nrhs, col0 + 4) : nrhs;
    int b = blockIdx.x;
    const int fb = xpass_fam_ctas(P.nq, P.fch);
    if (b < fb) {
        const int gw = b * 4 + (threadIdx.x >> 5);
        if (gw >= P.nq * P.fch) return;   // whole warps; the family work has no CTA barrier
        if (P.down) fam_dn32(gw / P.fch, gw % P.fch, P, col0, col1);
        else fam_up32(gw / P.fch, gw % P.fch, P, col0, col1, xsm32 + (threadIdx.x >> 5) * 4 * (2 * P.pS + 1));
    } else {
        b -= fb;
        translate32_dst(b / P.nch, b % P.nch, P, col0, col1, xsm32);
    }
}

// Dense scaled FP32 tables of one pass: W[m][n] = f_src(|m|) f_dst(|n|) V[n - m + pS + pD],
// f = s^|.| or s^-|.| as the expansion kind requires (up: multipoles M = M~ s^|m|,
// M~_n = M_n / s^|n|; down: locals L = L~ s^-|m|, L~_n = L_n s^|n|).
__global__ void k_xtab32(const XDst* __restrict__ dsts, const XSrc* __restrict__ srcs, const int* __restrict__ dlay,
                         const cd* __restrict__ xvec, const double* __restrict__ sc, int nlev, int lev_src,
                         int lev_dst, int down, const int64_t* __restrict__ wtab_off, cf* __restrict__ wtab) {
    const XDst d = dsts[blockIdx.x];
    const int lay = dlay[blockIdx.x];
    const double ss = sc[lay * nlev + lev_src], sd = sc[lay * nlev + lev_dst];
    const int ncD = 2 * d.p + 1;
    for (int j = d.src_begin; j < d.src_end; ++j) {
        const XSrc sr = srcs[j];
        const int ncS = 2 * sr.p + 1;
        const cd* V = xvec + sr.vec_off;
        for (int e = threadIdx.x; e < ncS * ncD; e += blockDim.x) {
            const int mi = e / ncD, ni = e - mi * ncD;
            const int m = mi - sr.p, nn = ni - d.p;
            const double f = down ? pow(ss, -(double)abs(m)) * pow(sd, (double)abs(nn))
                                  : pow(ss, (double)abs(m)) * pow(sd, -(double)abs(nn));
            const cd v = V[nn - m + sr.p + d.p];
            wtab[wtab_off[j] + e] = mkf((float)(f * v.x), (float)(f * v.y));
        }
    }
}

// Level hand-over between the FP32 and FP64 levels, over a coefficient range [c0, c0 + n) of
// every column (leading dimension ld), one launch for all columns: multipoles M = M~ s^|m| into
// FP64 (k_from32_cols), locals L~ += L s^|n| into FP32 (k_add_to32_cols; ispow = s^-|n|)
__global__ void k_from32_cols(const cf* __restrict__ in, const double* __restrict__ ispow, int64_t c0, int64_t n,
                              int nrhs, int64_t ld, cd* __restrict__ out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * nrhs;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = t / n, i = c0 + (t - col * n);
        const double f = 1.0 / ispow[i];   // multipoles: M = M~ s^|m|
        const cf v = in[col * ld + i];
        out[col * ld + i] = mk(f * (double)v.x, f * (double)v.y);
    }
}
__global__ void k_add_to32_cols(const cd* __restrict__ in, const double* __restrict__ ispow, int64_t c0, int64_t n,
                                int nrhs, int64_t ld, cf* __restrict__ out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * nrhs;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = t / n, i = c0 + (t - col * n);
        const double f = 1.0 / ispow[i];
        const cd v = in[col * ld + i];
        out[col * ld + i] = addf(out[col * ld + i], mkf((float)(f * v.x), (float)(f * v.y)));
    }
}

// ---------------------------------------------------------------------------
// replacing (in_flight: queued work may still read them) or releasing at destroy
// ------------------------------------------------------------------ coarse levels in double-float
// The coarse (wide-band) levels' M2L runs in double-float, with the same scales s as the FP32
// levels (the unscaled tables reach |H_2p(2 k w)| ~ 1e40 and more at orders near 75 in the
// low-k layers, past the FP32 exponent range).  The free-space sum
//     L_n = sum_m T_{m-n} M_m
// is split by the signs of n and m.  Where they differ (or m = 0), |m - n| = |m| + |n| and the
// scaled dense entry s^(|n| + |m|) T_{m-n} equals the scaled Toeplitz entry
// V~_{m-n} = s^|m-n| T_{m-n}: that half runs on (V~, M~) in scaled units.  Where they agree,
// |m - n| <= p and the unscaled T_{m-n} and M_m stay in range: that half runs unscaled.  So
// both halves keep the Toeplitz vectors (4p + 1 entries per table) and each lane of a slice
// takes one half per step: a slice's step q covers the opposite-sign half for q <= p and the
// same-sign half after.  The reaction part uses the dense scaled tables
// s_T^|m| s_S^|n| I_mn on scaled multipoles, as the FP32 levels do.  The results are summed
// and unscaled in FP64: L_n = s^-|n| (scaled sum) + (unscaled sum).

// scaled and unscaled double-float Toeplitz vectors of the listed free-space tables; amax
// collects the largest |component| stored (as float bits; non-finite values store +inf)
__device__ __forceinline__ void note_max(unsigned* amax, double a, double b) {
    double m = fmax(fabs(a), fabs(b));
    if (!(m <= 3.0e38)) m = 3.0e38 * 2.0;
    atomicMax(amax, __float_as_uint((float)m));
}
__global__ void k_ftab_df(const cd* __restrict__ m2lf, const int64_t* __restrict__ m2lf_off,
                          const int* __restrict__ list, const int* __restrict__ tab_p, const double* __restrict__ tab_s,
                          dfc* __restrict__ outs, dfc* __restrict__ outu, unsigned* __restrict__ amax) {
    const int id = list[blockIdx.x];
    const int p = tab_p[id];
    const double s = tab_s[id];
    const int64_t off = m2lf_off[id];
    for (int e = threadIdx.x; e <= 4 * p; e += blockDim.x) {
        const int j = abs(e - 2 * p);
        const cd v = m2lf[off + e];
        const double f = pow(s, (double)j);
        outs[off + e] = to_dfc(f * v.x, f * v.y);
        note_max(amax, f * v.x, f * v.y);
        if (j <= p) {
            outu[off + e] = to_dfc(v.x, v.y);
            note_max(amax, v.x, v.y);
        } else {
            outu[off + e] = dfc_zero();
        }
    }
}
// scaled double-float reaction tables of the listed keys (one CTA per key).  Each row m is
// further divided by 2^e_m, e_m the binary exponent of its largest scaled entry, so that every
// stored entry is below 1 in magnitude and a product with a scaled multipole stays inside the
// FP32 exponent range whatever the table's own growth; rsc[K.off + row] keeps 2^e_m, by which
// the M2L multiplies the row's sum (exactly: a power of two).
__global__ void k_rtab_df(const cd* __restrict__ m2lr, const ReactKey* __restrict__ keys, const int* __restrict__ list,
                          const double* __restrict__ key_ss, const double* __restrict__ key_st, dfc* __restrict__ out,
                          float* __restrict__ rsc, unsigned* __restrict__ amax) {
    const int kk = list[blockIdx.x];
    const ReactKey K = keys[kk];
    const int ncT = 2 * K.pT + 1, ncS = 2 * K.pS + 1;
    const double ss = key_ss[kk], st = key_st[kk];
    for (int mi = threadIdx.x; mi < ncT; mi += blockDim.x) {   // (m_out, n_in) at n_in ncT + m_out
        const double fm = pow(st, (double)abs(mi - K.pT));
        double mx = 0.0;
        for (int ni = 0; ni < ncS; ++ni) {
            const double f = fm * pow(ss, (double)abs(ni - K.pS));
            const cd v = m2lr[K.off + (int64_t)ni * ncT + mi];
            mx = fmax(mx, fmax(fabs(f * v.x), fabs(f * v.y)));
        }
        int e = 0;
        if (mx > 0.0 && mx <= 1e300) frexp(mx, &e);
        if (!(mx <= 1e300) || e > 120 || e < -120) {   // not representable: reported, never used
            note_max(amax, 1e300, 0.0);
            e = 0;
        }
        const double r = ldexp(1.0, -e);
        for (int ni = 0; ni < ncS; ++ni) {
            const double f = r * fm * pow(ss, (double)abs(ni - K.pS));
            const cd v = m2lr[K.off + (int64_t)ni * ncT + mi];
            out[K.off + (int64_t)ni * ncT + mi] = to_dfc(f * v.x, f * v.y);
        }
        rsc[K.off + mi] = ldexpf(1.0f, e);
        note_max(amax, mx, 0.0);
    }
}
// Per column, the binary exponent bound of the coarse levels' scaled multipoles (cells and
// reaction centres): emax[col] >= ilogb of every |component| of M ispow.  The double-float
// M2L divides that column by 2^(emax + 1), so its multipoles are below 1 in magnitude and its
// sums are bounded by the tables alone, whatever the scale of x.
__global__ void k_m_absmax(const cd* __restrict__ in, int64_t ld_in, const double* __restrict__ isp, int64_t c0,
                           int64_t n, int nrhs, int* __restrict__ emax) {
    int e = INT_MIN, col = -1;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * nrhs;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        const int64_t i = t - (int64_t)c * n;
        const cd v = in[(int64_t)c * ld_in + c0 + i];
        const double a = fmax(fabs(v.x), fabs(v.y)) * isp[c0 + i];
        if (c != col) {
            if (col >= 0 && e != INT_MIN) atomicMax(&emax[col], e);
            col = c;
            e = INT_MIN;
        }
        if (a > 0.0) e = max(e, min(ilogb(a), 2000));
    }
    if (col >= 0 && e != INT_MIN) atomicMax(&emax[col], e);
}
// the coarse levels' multipoles of every column as double-float, scaled (M ispow) and divided
// by 2^(emax + 1), and where outu is given also unscaled (M only divided by the same power of
// two); in: [cols][ld_in] from offset c0, out: [cols][n]
__global__ void k_m_to_df(const cd* __restrict__ in, int64_t ld_in, const double* __restrict__ isp, int64_t c0,
                          int64_t n, int nrhs, const int* __restrict__ emax, dfc* __restrict__ outs,
                          dfc* __restrict__ outu) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * nrhs;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = t / n, i = t - col * n;
        const cd v = in[col * ld_in + c0 + i];
        const int e = emax[col];
        const double r = (e < -2000) ? 1.0 : ldexp(1.0, -(e + 1));   // < -2000: an all-zero column
        const double f = isp[c0 + i] * r;
        outs[t] = to_dfc(f * v.x, f * v.y);
        if (outu) outu[t] = to_dfc(r * v.x, r * v.y);
    }
}

// M2L of the coarse levels in double-float: the work items, entry descriptors, index flips
// and partial-sum slots of the FP64 k_m2l (fmm_kernels.cuh).  Multipoles: Ms (scaled) and Mu
// (unscaled) of the boxes from coefficient c0, Mps (scaled) of the reaction centres from s0.
// Each thread turns its sums to unscaled FP64 before the slices are added in a fixed order;
// the outputs (L, reaction-centre locals, or partial sums for k_m2l_reduce) are FP64.
__global__ void __launch_bounds__(128) k_m2l_df(const M2LItem* __restrict__ items, const M2LEnt* __restrict__ ents,
                      const int* __restrict__ box_level, const int* __restrict__ p_level,
                      const int64_t* __restrict__ coef_off, const int* __restrict__ slot_of,
                      const int64_t* __restrict__ slot_coef, const dfc* __restrict__ fts,
                      const dfc* __restrict__ ftu, const int64_t* __restrict__ m2lf_off,
                      const dfc* __restrict__ rts, const float* __restrict__ rsc, const double* __restrict__ ispow,
                      int nrhs, int64_t ncoef,
                      int64_t nslotcoef, int nparts, const dfc* __restrict__ Ms, const dfc* __restrict__ Mu,
                      int64_t c0, int64_t ncd, const dfc* __restrict__ Mps, int64_t s0, int64_t nsd,
                      const int* __restrict__ emax, cd* __restrict__ Lout, cd* __restrict__ Lp,
                      cd* __restrict__ part) {
    __shared__ cd red[3 * 128];
    __shared__ M2LEnt se[64];
    const M2LItem it = items[blockIdx.x];
    const int T = it.box;
    const int p = p_level[box_level[T]];
    const int nco = 2 * p + 1;
    const int W = it.w, NS = 128 / W;
    const int lane = threadIdx.x % W, sl = threadIdx.x / W;
    const int idx = it.chunk * W + lane;
    const bool live = sl < NS && idx < nco;
    const int nn = idx - p;
    const int sg = nn >= 0 ? 1 : -1;
    const double isp = live ? ispow[coef_off[T] + idx] : 0.0;   // s^-|n| of the target box
    const int cpb = (nrhs + gridDim.y - 1) / gridDim.y;   // blockIdx.y: a group of columns
    const int col0 = blockIdx.y * cpb, col1 = min(nrhs, col0 + cpb);
    for (int col = col0; col < col1; ++col) {
        const dfc* Msc = Ms + (int64_t)col * ncd - c0 + p;    // [E.src + m] is M~_m of the source box
        const dfc* Muc = Mu + (int64_t)col * ncd - c0 + p;
        const dfc* Mpc = Mps + (int64_t)col * nsd - s0;
        const dfc* Mbc = Ms + (int64_t)col * ncd - c0;
        dfc acc0 = dfc_zero(), acc1 = dfc_zero(), acc2 = dfc_zero(), accu = dfc_zero();
        for (int eb = it.e0; eb < it.e1; eb += 64) {
            const int cnt = min(64, it.e1 - eb);
            __syncthreads();
            if (threadIdx.x < cnt) se[threadIdx.x] = ents[eb + threadIdx.x];
            __syncthreads();
            if (!live) continue;
            for (int q = 0; q < cnt; ++q) {
                const M2LEnt E = se[q];
                if (!(E.flags & M2L_REACT)) {
                    const int64_t tb = m2lf_off[E.tab] + 2 * p - nn;   // [tb + m] is entry m - n
                    const dfc* ms_ = Msc + E.src;
                    const dfc* mu_ = Muc + E.src;
                    for (int k = sl; k < nco; k += NS) {
                        if (k <= p) {
                            const int m = -sg * k;
                            dfc_fma(acc0, ms_[m], fts[tb + m]);
                        } else {
                            const int m = sg * (k - p);
                            dfc_fma(accu, mu_[m], ftu[tb + m]);
                        }
                    }
                } else {
                    const dfc* src = (E.flags & M2L_SRC_SLOT) ? Mpc + E.src : Mbc + E.src;
                    const bool bdown = (E.flags & M2L_B_DOWN) != 0;
                    const int mrow = bdown ? nn : -nn;
                    const bool flip = (E.flags & M2L_FLIP) != 0;
                    const int row = flip ? p - mrow : p + mrow;
                    const dfc* col_m = rts + E.tab + row + (flip ? (int64_t)2 * p * nco : 0);
                    const int64_t cs = flip ? -(int64_t)nco : (int64_t)nco;
                    dfc bsum = dfc_zero();
                    if (E.flags & M2L_A_DOWN) {
                        for (int mi = sl; mi < nco; mi += NS) dfc_fma(bsum, col_m[mi * cs], src[mi]);
                    } else {
                        for (int mi = sl; mi < nco; mi += NS) dfc_fma(bsum, col_m[mi * cs], dfc_sign(src[2 * p - mi], mi - p));
                    }
                    const float rf = rsc[E.tab + row];
                    bsum = dfc_sign(make_float4(bsum.x * rf, bsum.y * rf, bsum.z * rf, bsum.w * rf), (!bdown) & mrow);
                    const int dst = (E.flags >> M2L_DST_SHIFT) & 3;
                    if (dst == 0) dfc_add(acc0, bsum);
                    else if (dst == 1) dfc_add(acc1, bsum);
                    else dfc_add(acc2, bsum);
                }
            }
        }
        if (sl < NS) {
            const int ecol = emax[col];
            const double unit = (ecol < -2000) ? 1.0 : ldexp(1.0, ecol + 1);   // the column's normalisation
            const double f = isp * unit;
            red[(0 * NS + sl) * W + lane] = mk(fma(f, df_value(acc0.x, acc0.y), unit * df_value(accu.x, accu.y)),
                                               fma(f, df_value(acc0.z, acc0.w), unit * df_value(accu.z, accu.w)));
            red[(1 * NS + sl) * W + lane] = mk(f * df_value(acc1.x, acc1.y), f * df_value(acc1.z, acc1.w));
            red[(2 * NS + sl) * W + lane] = mk(f * df_value(acc2.x, acc2.y), f * df_value(acc2.z, acc2.w));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * W; i += blockDim.x) {
            const int k = i / W, ln = i - k * W, ix = it.chunk * W + ln;
            if (ix >= nco) continue;
            cd v = red[(k * NS) * W + ln];
            for (int q = 1; q < NS; ++q) v += red[(k * NS + q) * W + ln];
            if (it.part >= 0) {
                part[(((int64_t)col * nparts + it.part) * 3 + k) * XT_W + ln] = v;
            } else {
                const int ts = (k == 0) ? -1 : slot_of[2 * T + k - 1];
                if (k == 0) Lout[(int64_t)col * ncoef + coef_off[T] + ix] = v;
                else if (ts >= 0) Lp[(int64_t)col * nslotcoef + slot_coef[ts] + ix] = v;
            }
        }
        __syncthreads();
    }
}

static void mixed_free_buffers(MixedState* ms, bool in_flight) {
    void* bufs[5] = {ms->M, ms->L, ms->Mp, ms->Lp, ms->part};
    for (void* b : bufs) {
        if (in_flight) dev_release_now(b);
        else dev_release(b);
    }
    ms->M = ms->L = ms->Mp = ms->Lp = ms->part = nullptr;
    ms->cols = 0;
}
static void mixed_free_df(MixedState* ms, bool in_flight) {
    for (void* b : {(void*)ms->Mdf, (void*)ms->Mudf, (void*)ms->Mpdf, (void*)ms->df_emax}) {
        if (in_flight) dev_release_now(b);
        else dev_release(b);
    }
    ms->Mdf = ms->Mudf = ms->Mpdf = nullptr;
    ms->df_emax = nullptr;
    ms->df_cols = 0;
}

void mixed_destroy(lfmm_geometry_s* g) {
    if (!g->mixed) return;
    MixedState* ms = g->mixed;
    mixed_free_buffers(ms, false);
    mixed_free_df(ms, false);
    dev_release(ms->ftab_df); dev_release(ms->rtab_df); dev_release(ms->rtab_rsc);
    dev_release(ms->ispow); dev_release(ms->ispow_slot); dev_release(ms->ftab); dev_release(ms->ftab_off);
    dev_release(ms->rtab); dev_release(ms->d_scale); dev_release(ms->wtab); dev_release(ms->wtab_off);
    dev_release(ms->d_xd_layer);
    dev_release(ms->qoff); dev_release(ms->q_bd); dev_release(ms->q_bs); dev_release(ms->q_blay);
    dev_release(ms->q_bwoff);
    dev_release(ms->tc_boxes); dev_release(ms->tc_ent_ptr); dev_release(ms->tc_err);
    if (ms->tc_err_host) cudaFreeHost(ms->tc_err_host);
    delete ms;
    g->mixed = nullptr;
}

template <typename T>
static T* upload_raw(const std::vector<T>& v, size_t& bytes) {
    T* p = nullptr;
    const size_t b = sizeof(T) * std::max<size_t>(v.size(), 1);
    cuda_check(cudaMallocAsync((void**)&p, b, cudaStreamPerThread), "cudaMallocAsync (precision form)");
    bytes += b;
    if (!v.empty())
        cuda_check(cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, cudaStreamPerThread),
                   "upload");
    return p;
}

// coefficient ranges of one level: boxes, then reaction centres (both follow box order)
static void level_ranges(lfmm_geometry_s* g, int l, int64_t* c0, int64_t* c1, int64_t* s0, int64_t* s1) {
    const TreeHost& t = g->tree;
    *c0 = g->box_coef_off_host[t.level_start[l]];
    *c1 = (l < t.D) ? g->box_coef_off_host[t.level_start[l + 1]] : g->ncoef;
    *s0 = g->nslotcoef;
    *s1 = g->nslotcoef;
    for (size_t q = 0; q < g->slot_box_host.size(); ++q) {
        const int lv = t.box_level[g->slot_box_host[q]];
        if (lv >= l && *s0 == g->nslotcoef) *s0 = g->slot_coef_host[q];
        if (lv > l) { *s1 = g->slot_coef_host[q]; break; }
    }
    if (*s1 < *s0) *s1 = *s0;
}

// Scales and FP32 tables of the precision form (once per geometry, on first use).
static void mixed_build(lfmm_geometry_s* g) {
    TreeHost& t = g->tree;
    const int D = t.D, l0 = t.l0, nlev = D + 1, nl = g->m.nl;
    MixedState* ms = new MixedState();
    g->mixed = ms;
    ms->scale.assign((size_t)nl * nlev, 1.0);
    for (int lay = 0; lay < nl; ++lay)
        for (int l = l0; l <= D; ++l)
            ms->scale[lay * nlev + l] = choose_scale(g->m.k[lay], t.width(l), t.p_level[l]);
    // s^-|n| per coefficient of every box and reaction centre
    std::vector<double> isp((size_t)std::max<int64_t>(g->ncoef, 1), 1.0);
    for (int b = t.level_start[l0]; b < t.nbox; ++b) {
        const int l = t.box_level[b], p = t.p_level[l];
        const double s = ms->scale[t.box_layer[b] * nlev + l];
        for (int i = 0; i <= 2 * p; ++i) isp[g->box_coef_off_host[b] + i] = std::pow(s, -(double)std::abs(i - p));
    }
    std::vector<double> isps((size_t)std::max<int64_t>(g->nslotcoef, 1), 1.0);
    for (size_t q = 0; q < g->slot_box_host.size(); ++q) {
        const int b = g->slot_box_host[q];
        const int l = t.box_level[b], p = t.p_level[l];
        const double s = ms->scale[t.box_layer[b] * nlev + l];
        for (int i = 0; i <= 2 * p; ++i) isps[g->slot_coef_host[q] + i] = std::pow(s, -(double)std::abs(i - p));
    }
    ms->ispow = upload_raw(isp, ms->bytes);
    ms->ispow_slot = upload_raw(isps, ms->bytes);
    // free-space tables
    const int ntab = (int)g->ftab_lay.size();
    std::vector<int> tp(ntab);
    std::vector<double> ts(ntab);
    std::vector<int64_t> off32(ntab);
    int64_t tot = 0;
    for (int id = 0; id < ntab; ++id) {
        const int l = g->ftab_lev[id];
        tp[id] = t.p_level[l];
        ts[id] = ms->scale[g->ftab_lay[id] * nlev + l];
        off32[id] = tot;
        tot += (int64_t)(2 * tp[id] + 1) * (2 * tp[id] + 1);
    }
    size_t scratch = 0;
    int* d_tp = upload_raw(tp, scratch);
    double* d_ts = upload_raw(ts, scratch);
    ms->ftab_off = upload_raw(off32, ms->bytes);
    cuda_check(cudaMallocAsync((void**)&ms->ftab, sizeof(cf) * std::max<int64_t>(tot, 1), cudaStreamPerThread),
               "cudaMallocAsync ftab32");
    ms->bytes += sizeof(cf) * std::max<int64_t>(tot, 1);
    if (ntab > 0) k_free32_tables<<<ntab, 256>>>(g->d_m2lf, g->d_m2lf_off, d_tp, d_ts, ms->ftab_off, ms->ftab);
    cuda_check(cudaGetLastError(), "k_free32_tables");
    // reaction tables
    const int nk = (int)g->rkeys_host.size();
    int64_t rtot = 0;
    std::vector<double> kss(nk), kst(nk);
    for (int kk = 0; kk < nk; ++kk) {
        const ReactKey& K = g->rkeys_host[kk];
        rtot = std::max<int64_t>(rtot, K.off + (int64_t)(2 * K.pT + 1) * (2 * K.pS + 1));
        kss[kk] = ms->scale[g->rkey_lay_s[kk] * nlev + K.level];
        kst[kk] = ms->scale[g->rkey_lay_t[kk] * nlev + K.level];
    }
    double* d_kss = upload_raw(kss, scratch);
    double* d_kst = upload_raw(kst, scratch);
    cuda_check(cudaMallocAsync((void**)&ms->rtab, sizeof(cf) * std::max<int64_t>(rtot, 1), cudaStreamPerThread),
               "cudaMallocAsync rtab32");
    ms->bytes += sizeof(cf) * std::max<int64_t>(rtot, 1);
    if (nk > 0) k_react32_tables<<<nk, 256>>>(g->d_m2lr, g->d_rkeys, d_kss, d_kst, ms->rtab);
    // dense scaled tables of the FP32 M2M passes (parents at levels >= lm) and L2L
    // passes (children at levels > lm)
    ms->lm = std::max(l0, std::min(mixed_level(g), D + 1));
    ms->d_scale = upload_raw(ms->scale, ms->bytes);
    if (ms->lm > l0) {
        // Double-float tables of the coarse levels' M2L.  They are used when every stored
        // component stays below 1e13 and the scaled multipole basis below 1e13 (log10 sum at
        // most 26): products then stay below 1e26 times the sources' total |weight x|,
        // far inside the FP32 exponent range.  Otherwise those levels keep the FP64 M2L.
        double big_m = 0.0;
        for (int lay = 0; lay < nl; ++lay)
            for (int l = l0; l < ms->lm; ++l) {
                double bm = 0.0;
                choose_scale(g->m.k[lay], t.width(l), t.p_level[l], &bm);
                big_m = std::max(big_m, bm);
            }
        std::vector<int> ftl, rkl;
        for (int id = 0; id < ntab; ++id)
            if (g->ftab_lev[id] < ms->lm) ftl.push_back(id);
        for (int kk = 0; kk < nk; ++kk)
            if (g->rkeys_host[kk].level < ms->lm) rkl.push_back(kk);
        const int64_t flen = std::max<int64_t>(g->m2lf_len, 1);
        cuda_check(cudaMallocAsync((void**)&ms->ftab_df, sizeof(dfc) * 2 * flen, cudaStreamPerThread),
                   "cudaMallocAsync ftab_df");
        cuda_check(cudaMallocAsync((void**)&ms->rtab_df, sizeof(dfc) * std::max<int64_t>(rtot, 1), cudaStreamPerThread),
                   "cudaMallocAsync rtab_df");
        cuda_check(cudaMallocAsync((void**)&ms->rtab_rsc, sizeof(float) * std::max<int64_t>(rtot, 1),
                                   cudaStreamPerThread), "cudaMallocAsync rtab_rsc");
        unsigned* d_amax = nullptr;   // [2]: free-space, reaction
        cuda_check(cudaMallocAsync((void**)&d_amax, 2 * sizeof(unsigned), cudaStreamPerThread), "cudaMallocAsync amax");
        cuda_check(cudaMemsetAsync(d_amax, 0, 2 * sizeof(unsigned), cudaStreamPerThread), "amax reset");
        if (!ftl.empty()) {
            int* d_l = upload_raw(ftl, scratch);
            k_ftab_df<<<(int)ftl.size(), 256, 0, cudaStreamPerThread>>>(g->d_m2lf, g->d_m2lf_off, d_l, d_tp, d_ts,
                                                                        ms->ftab_df, ms->ftab_df + flen, d_amax);
            cuda_check(cudaGetLastError(), "k_ftab_df");
            dev_release(d_l);
        }
        if (!rkl.empty()) {
            int* d_l = upload_raw(rkl, scratch);
            k_rtab_df<<<(int)rkl.size(), 256, 0, cudaStreamPerThread>>>(g->d_m2lr, g->d_rkeys, d_l, d_kss, d_kst,
                                                                        ms->rtab_df, ms->rtab_rsc, d_amax + 1);
            cuda_check(cudaGetLastError(), "k_rtab_df");
            dev_release(d_l);
        }
        unsigned amax_bits[2] = {0, 0};
        cuda_check(cudaMemcpyAsync(amax_bits, d_amax, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost,
                                   cudaStreamPerThread), "amax read");
        cuda_check(cudaStreamSynchronize(cudaStreamPerThread), "double-float tables");
        dev_release(d_amax);
        float amax[2];
        std::memcpy(amax, amax_bits, sizeof(amax));
        for (int i = 0; i < 2; ++i)
            ms->df_range[i] = std::isfinite(amax[i]) ? std::log10(std::max(amax[i], 1e-30f)) : 1e300;
        ms->df_range[2] = big_m;
        // The multipoles enter normalised below 1 (per column) and the reaction rows are stored
        // below 1 with their own factors, so every product is bounded by the free-space tables;
        // those must stay far inside the FP32 range (and the reaction rows' factors within it).
        ms->df_ok = ms->df_range[1] <= 1e299 && ms->df_range[0] <= 20.0;
        if (ms->df_ok) {
            ms->bytes += sizeof(dfc) * (2 * flen + std::max<int64_t>(rtot, 1)) + sizeof(float) * std::max<int64_t>(rtot, 1);
            int64_t d0, d1, e0, e1;
            level_ranges(g, l0, &ms->df_c0, &d1, &ms->df_s0, &e1);
            level_ranges(g, ms->lm - 1, &d0, &d1, &e0, &e1);
            ms->df_ncd = d1 - ms->df_c0;
            ms->df_nsd = e1 - ms->df_s0;
        } else {
            dev_release(ms->ftab_df);
            dev_release(ms->rtab_df);
            dev_release(ms->rtab_rsc);
            ms->ftab_df = ms->rtab_df = nullptr;
            ms->rtab_rsc = nullptr;
        }
    }
    {   // the tensor-core M2L's boxes: every box of the FP32 levels
        std::vector<int> tb;
        for (int b = (ms->lm <= D ? t.level_start[ms->lm] : t.nbox); b < t.nbox; ++b) tb.push_back(b);
        ms->n_tc_boxes = (int)tb.size();
        ms->tc_boxes = upload_raw(tb, ms->bytes);
        ms->tc_ent_ptr = upload_raw(g->m2l_ent_ptr_host, ms->bytes);
        ms->tc_p = ms->lm <= D ? t.p_level[ms->lm] : 0;
        const std::vector<int> zero(1, 0);
        ms->tc_err = upload_raw(zero, ms->bytes);
        cuda_check(cudaMallocHost((void**)&ms->tc_err_host, sizeof(int)), "cudaMallocHost");
        *ms->tc_err_host = 0;
    }
    ms->d_xd_layer = upload_raw(g->xd_layer_host, ms->bytes);
    std::vector<int64_t> woff(std::max<size_t>(g->xsrc_host.size(), 1), -1);
    int64_t wtot = 0;
    auto plan = [&](int b0, int b1) {
        for (int i = b0; i < b1; ++i) {
            const XDst& d = g->xdst_host[i];
            for (int j = d.src_begin; j < d.src_end; ++j) {
                woff[j] = wtot;
                wtot += (int64_t)(2 * d.p + 1) * (2 * g->xsrc_host[j].p + 1);
            }
        }
    };
    for (int lp = D - 1; lp >= ms->lm; --lp) plan(g->up_begin[lp], g->up_end[lp]);
    for (int l = ms->lm + 1; l <= D; ++l) plan(g->dn_begin[l], g->dn_end[l]);
    // cell families of the FP32 passes (child levels lm + 1 .. D): a base table per
    // (level, pass, layer), record i = ((l - lm - 1) 2 + down) nl + layer
    std::vector<XDst> bd;
    std::vector<XSrc> bs;
    std::vector<int> blay;
    std::vector<int64_t> bwoff, qoff((size_t)(nlev + 1) * 2 * nl, -1);
    for (int l = ms->lm + 1; l <= D; ++l)
        for (int down = 0; down < 2; ++down)
            for (int lay = 0; lay < nl; ++lay) {
                const int pS = down ? t.p_level[l - 1] : t.p_level[l], pD = down ? t.p_level[l] : t.p_level[l - 1];
                const int i = (int)bd.size();
                bd.push_back(XDst{0, pD, 0, i, i + 1});
                bs.push_back(XSrc{0, g->qvec_host[(size_t)(lay * nlev + l) * 2 + down], pS, 0});
                blay.push_back(lay);
                bwoff.push_back(wtot);
                qoff[(size_t)(l * 2 + down) * nl + lay] = wtot;
                wtot += (int64_t)(2 * pD + 1) * (2 * pS + 1);
            }
    ms->qoff = upload_raw(qoff, ms->bytes);
    ms->q_bd = upload_raw(bd, ms->bytes);
    ms->q_bs = upload_raw(bs, ms->bytes);
    ms->q_blay = upload_raw(blay, ms->bytes);
    ms->q_bwoff = upload_raw(bwoff, ms->bytes);
    ms->wtab_off = upload_raw(woff, ms->bytes);
    cuda_check(cudaMallocAsync((void**)&ms->wtab, sizeof(cf) * std::max<int64_t>(wtot, 1), cudaStreamPerThread),
               "cudaMallocAsync pass tables 32");
    ms->bytes += sizeof(cf) * std::max<int64_t>(wtot, 1);
    for (int lp = D - 1; lp >= ms->lm; --lp) {
        const int nd = g->up_end[lp] - g->up_begin[lp];
        if (nd > 0)
            k_xtab32<<<nd, 256>>>(g->d_xdst + g->up_begin[lp], g->d_xsrc, ms->d_xd_layer + g->up_begin[lp], g->d_xvec,
                                  ms->d_scale, nlev, lp + 1, lp, 0, ms->wtab_off, ms->wtab);
    }
    for (int l = ms->lm + 1; l <= D; ++l) {
        const int nd = g->dn_end[l] - g->dn_begin[l];
        if (nd > 0)
            k_xtab32<<<nd, 256>>>(g->d_xdst + g->dn_begin[l], g->d_xsrc, ms->d_xd_layer + g->dn_begin[l], g->d_xvec,
                                  ms->d_scale, nlev, l - 1, l, 1, ms->wtab_off, ms->wtab);
        for (int down = 0; down < 2; ++down) {
            const int b0 = ((l - ms->lm - 1) * 2 + down) * nl;
            k_xtab32<<<nl, 256>>>(ms->q_bd + b0, ms->q_bs, ms->q_blay + b0, g->d_xvec, ms->d_scale, nlev,
                                  down ? l - 1 : l, down ? l : l - 1, down, ms->q_bwoff, ms->wtab);
        }
    }
    cuda_check(cudaGetLastError(), "k_xtab32");
    // shared memory of the FP32 P2M / L2P (all entries at the leaf order)
    const int pD = t.p_level[D], gp = g->group_max_pts, ge = g->group_max_ent;
    const int rs_p2m = g->combined ? 2 * pD + 3 : pD + 1;   // basis row length (k_p2m32)
    ms->smem_p2m = (size_t)gp * rs_p2m * sizeof(cf) + (size_t)gp * sizeof(cf) + (size_t)(gp + 1) * sizeof(int);
    ms->smem_l2p = ((size_t)gp * (pD + 1) + 1) * sizeof(float) + (size_t)ge * (2 * pD + 1) * sizeof(cf);
    raise_smem_limit((const void*)k_p2m32, ms->smem_p2m, "p2m32 smem");
    raise_smem_limit((const void*)k_l2p32, ms->smem_l2p, "l2p32 smem");
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(cudaStreamPerThread);
    dev_release(d_tp); dev_release(d_ts); dev_release(d_kss); dev_release(d_kst);
    cuda_check(e1, "k_react32_tables");
    cuda_check(e2, "precision form tables");
}

// First level whose far field runs in FP32: the levels whose expansion order is
// at most 1.5 p, i.e. the wide-band rule raised it little.  On coarser levels
// (boxes many wavelengths wide, orders 2-3 times p) the local coefficients of
// orders well above k rho reach 1e8 and more relative to the field, FP32
// carries them to about 1e-4, and the local-to-local translations pass those
// absolute errors down the tree; there the FP64 kernels stay.  (C2: orders 25
// and 20 run in FP32, 37 and 57 in FP64; operator difference 2.9e-7.)
int mixed_level(lfmm_geometry_s* g) {
    const TreeHost& t = g->tree;
    for (int l = t.l0; l <= t.D; ++l)
        if (2 * t.p_level[l] <= 3 * g->p) return l;
    return t.D + 1;
}

void mixed_setup(lfmm_geometry_s* g, int nrhs) {
    if (!g->mixed) mixed_build(g);
    MixedState* ms = g->mixed;
    if (ms->cols < nrhs) {
        mixed_free_buffers(ms, true);
        const size_t nc = (size_t)std::max<int64_t>(g->ncoef, 1) * nrhs;
        const size_t ns = (size_t)std::max<int64_t>(g->nslotcoef, 1) * nrhs;
        ms->M = (cf*)dev_alloc_ready(sizeof(cf) * nc, "M32");
        ms->L = (cf*)dev_alloc_ready(sizeof(cf) * nc, "L32");
        ms->Mp = (cf*)dev_alloc_ready(sizeof(cf) * ns, "Mp32");
        ms->Lp = (cf*)dev_alloc_ready(sizeof(cf) * ns, "Lp32");
        ms->part = (cf*)dev_alloc_ready(sizeof(cf) * (size_t)std::max(g->n_m2l_parts, 1) * 3 * XT_W * nrhs,
                                        "M2L partial sums 32");
        ms->cols = nrhs;
    }
}

void mixed_p2m(lfmm_geometry_s* g, const cd* x_sorted, int nrhs, cudaStream_t s) {
    MixedState* ms = g->mixed;
    const int D = g->tree.D, nlev = D + 1;
    k_p2m32<<<g->n_leaf_groups, 128, ms->smem_p2m, s>>>(g->d_leaf_groups, g->d_leaf_entries, g->m, ms->d_scale, D, nlev,
                                                       g->d_x, g->d_y, g->d_w, g->d_nx, g->d_ny, x_sorted, g->n,
                                                       nrhs, g->ncoef, ms->M);
    cuda_check(cudaGetLastError(), "k_p2m32");
    ++g->n_launches;
    if (g->n_slot_groups > 0) {
        k_p2m32<<<g->n_slot_groups, 128, ms->smem_p2m, s>>>(g->d_slot_groups, g->d_slot_entries, g->m, ms->d_scale, D,
                                                           nlev, g->d_x, g->d_y, g->d_w, g->d_nx, g->d_ny,
                                                           x_sorted, g->n, nrhs, g->nslotcoef, ms->Mp);
        cuda_check(cudaGetLastError(), "k_p2m32 slots");
        ++g->n_launches;
    }
}

// one FP32 level pass: M2M into the parents at level - 1 (down = 0) or L2L into the
// children at level (down = 1)
static void pass32(lfmm_geometry_s* g, int level, int down, int nrhs, cudaStream_t s) {
    MixedState* ms = g->mixed;
    const TreeHost& t = g->tree;
    XPass32 P;
    P.dsts = g->d_xdst + (down ? g->dn_begin[level] : g->up_begin[level - 1]);
    P.srcs = g->d_xsrc;
    P.wtab_off = ms->wtab_off;
    P.wtab = ms->wtab;
    P.qx = g->d_qx + g->q_begin[level];
    P.qoff = ms->qoff + (size_t)(level * 2 + down) * g->m.nl;
    P.nq = g->q_end[level] - g->q_begin[level];
    P.nd = down ? g->dn_end[level] - g->dn_begin[level] : g->up_end[level - 1] - g->up_begin[level - 1];
    P.pS = down ? t.p_level[level - 1] : t.p_level[level];
    P.pD = down ? t.p_level[level] : t.p_level[level - 1];
    // FP32 translations are not bound by an arithmetic pipe: 16-lane chunks (more CTAs)
    // measured faster here than rows as wide as the coefficient count
    const int nco = 2 * P.pD + 1;
    P.w = XT_W;
    P.nch = (nco + P.w - 1) / P.w;
    xpass_fam_split(P.nq, P.pD, &P.fch, &P.fr);
    P.down = down;
    P.accumulate = down;   // M2M writes, L2L adds to the FP32 M2L's locals
    P.ncoef = g->ncoef;
    P.nslotcoef = g->nslotcoef;
    P.X = down ? ms->L : ms->M;
    P.Xp = down ? ms->Lp : ms->Mp;
    const int items = xpass_fam_ctas(P.nq, P.fch) + P.nd * P.nch;
    if (items == 0) return;
    const size_t smem = sizeof(cf) * (size_t)std::max(128, down ? 0 : 16 * (2 * P.pS + 1));
    const int ng = col_groups(nrhs);
    dim3 grid(items, 1, ng);
    if (ng > 1) {
        raise_smem_limit((const void*)k_translate32<true>, smem, "translate32 smem");
        k_translate32<true><<<grid, 128, smem, s>>>(P, nrhs);
    } else {
        raise_smem_limit((const void*)k_translate32<false>, smem, "translate32 smem");
        k_translate32<false><<<grid, 128, smem, s>>>(P, nrhs);
    }
    cuda_check(cudaGetLastError(), "k_translate32");
    ++g->n_launches;
}

void mixed_m2m(lfmm_geometry_s* g, int lp, int nrhs, cudaStream_t s) { pass32(g, lp + 1, 0, nrhs, s); }

void mixed_l2l(lfmm_geometry_s* g, int l, int nrhs, cudaStream_t s) { pass32(g, l, 1, nrhs, s); }


void mixed_m_to64(lfmm_geometry_s* g, int l, int nrhs, cudaStream_t s) {
    MixedState* ms = g->mixed;
    int64_t c0, c1, s0, s1;
    level_ranges(g, l, &c0, &c1, &s0, &s1);
    if (c1 > c0) {
        const int64_t n = (c1 - c0) * nrhs;
        k_from32_cols<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(
            ms->M, ms->ispow, c0, c1 - c0, nrhs, g->ncoef, g->d_M);
        ++g->n_launches;
    }
    if (s1 > s0) {
        const int64_t n = (s1 - s0) * nrhs;
        k_from32_cols<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(
            ms->Mp, ms->ispow_slot, s0, s1 - s0, nrhs, g->nslotcoef, g->d_Mp);
        ++g->n_launches;
    }
    cuda_check(cudaGetLastError(), "k_from32_cols");
}

void mixed_l_add(lfmm_geometry_s* g, int l, int nrhs, cudaStream_t s) {
    MixedState* ms = g->mixed;
    int64_t c0, c1, s0, s1;
    level_ranges(g, l, &c0, &c1, &s0, &s1);
    if (c1 > c0) {
        const int64_t n = (c1 - c0) * nrhs;
        k_add_to32_cols<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(
            g->d_L, ms->ispow, c0, c1 - c0, nrhs, g->ncoef, ms->L);
        ++g->n_launches;
    }
    if (s1 > s0) {
        const int64_t n = (s1 - s0) * nrhs;
        k_add_to32_cols<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(
            g->d_Lp, ms->ispow_slot, s0, s1 - s0, nrhs, g->nslotcoef, ms->Lp);
        ++g->n_launches;
    }
    cuda_check(cudaGetLastError(), "k_add_to32_cols");
}

void mixed_l2p(lfmm_geometry_s* g, cd* y_sorted, int nrhs, cudaStream_t s) {
    MixedState* ms = g->mixed;
    const int D = g->tree.D, nlev = D + 1;
    k_l2p32<<<g->n_leaf_groups, 128, ms->smem_l2p, s>>>(g->d_leaf_groups, g->d_leaf_entries, g->m, ms->d_scale, D, nlev,
                                                       g->d_x, g->d_y, g->n, nrhs, g->ncoef, ms->L, y_sorted);
    cuda_check(cudaGetLastError(), "k_l2p32");
    ++g->n_launches;
    if (g->n_slot_groups > 0) {
        k_l2p32<<<g->n_slot_groups, 128, ms->smem_l2p, s>>>(g->d_slot_groups, g->d_slot_leaf_entries, g->m,
                                                           ms->d_scale, D, nlev, g->d_x, g->d_y, g->n, nrhs,
                                                           g->nslotcoef, ms->Lp, y_sorted);
        cuda_check(cudaGetLastError(), "k_l2p32 slots");
        ++g->n_launches;
    }
}

// M2L of the precision form on the levels >= min_level (their multipoles are FP32 already).
// The tensor-core path: many columns (TC_MIN_COLS or more), every FP32 level at
// an order whose real-form rows 2(2p+1) fit one 128-row MMA.
#define TC_MIN_COLS 16
static bool m2l_tc(lfmm_geometry_s* g, int nrhs, int min_level, cudaStream_t s) {
    MixedState* ms = g->mixed;
    const int nco = 2 * ms->tc_p + 1;
    if (nrhs < TC_MIN_COLS || g->m2l_simt || ms->n_tc_boxes == 0 || 2 * nco > 128 || min_level != ms->lm)
        return false;
    mixed_check_waits(g);
    // K: real part at 0, imaginary part at kh = nco rounded up to 4 (16-byte stores), padded to 8
    const int kp = (2 * ((nco + 3) / 4 * 4) + 7) / 8 * 8;
    for (int c0 = 0; c0 < nrhs; c0 += TC_MAXN) {
        const int nc = std::min(TC_MAXN, nrhs - c0);
        const int np = nc <= 16 ? 16 : 32;
        const size_t smem = (size_t)(2 * 128 + 2 * np) * kp * sizeof(float);
        auto kern = np == 16 ? k_m2l32_tc<16> : k_m2l32_tc<32>;
        raise_smem_limit((const void*)kern, smem, "m2l tc smem");
        kern<<<ms->n_tc_boxes, 128, smem, s>>>(ms->tc_boxes, ms->tc_ent_ptr, g->d_m2l_ents, g->d_box_level,
                                               g->d_p_level, g->d_coef_off, g->d_slot_of, g->d_slot_coef, ms->ftab,
                                               ms->ftab_off, ms->rtab, c0, nc, kp, g->ncoef, g->nslotcoef, ms->M,
                                               ms->Mp, ms->L, ms->Lp, ms->tc_err);
        cuda_check(cudaGetLastError(), "k_m2l32_tc");
        ++g->n_launches;
    }
    cuda_check(cudaMemcpyAsync(ms->tc_err_host, ms->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s), "tc status");
    return true;
}

void mixed_check_waits(lfmm_geometry_s* g) {
    MixedState* ms = g->mixed;
    if (!ms || !ms->tc_err_host || *ms->tc_err_host == 0) return;
    // no launch of this geometry is in flight that could set it again (the caller's
    // stream has been synchronised, or the status is from an earlier call's)
    cuda_check(cudaMemsetAsync(ms->tc_err, 0, sizeof(int), cudaStreamPerThread), "tc status reset");
    cuda_check(cudaStreamSynchronize(cudaStreamPerThread), "tc status reset");
    *ms->tc_err_host = 0;
    throw TimeoutError{"tensor-core M2L: an mbarrier wait gave up; that product's M2L contributions were zeroed"};
}

bool mixed_coarse_df(lfmm_geometry_s* g) { return g->mixed && g->mixed->df_ok; }
void mixed_info(lfmm_geometry_s* g, int* lm, int* df, double* range) {
    *lm = g->mixed ? g->mixed->lm : std::max(g->tree.l0, std::min(mixed_level(g), g->tree.D + 1));
    *df = g->mixed ? (g->mixed->df_ok ? 1 : 0) : -1;
    for (int i = 0; i < 3; ++i) range[i] = g->mixed ? g->mixed->df_range[i] : 0.0;
}

void mixed_m2l_coarse(lfmm_geometry_s* g, int nrhs, int n_items, cudaStream_t s) {
    MixedState* ms = g->mixed;
    if (n_items <= 0) return;
    if (ms->df_cols < nrhs) {
        mixed_free_df(ms, true);
        const size_t nc = (size_t)std::max<int64_t>(ms->df_ncd, 1) * nrhs;
        ms->Mdf = (dfc*)dev_alloc_ready(sizeof(dfc) * nc, "M double-float");
        ms->Mudf = (dfc*)dev_alloc_ready(sizeof(dfc) * nc, "M double-float");
        ms->Mpdf = (dfc*)dev_alloc_ready(sizeof(dfc) * (size_t)std::max<int64_t>(ms->df_nsd, 1) * nrhs,
                                         "reaction-centre M double-float");
        ms->df_emax = (int*)dev_alloc_ready(sizeof(int) * nrhs, "column exponents");
        ms->df_cols = nrhs;
    }
    // every column's exponent bound over its coarse multipoles (cells and reaction centres)
    cuda_check(cudaMemsetAsync(ms->df_emax, 0x80, sizeof(int) * nrhs, s), "exponent reset");   // 0x80808080: none
    if (ms->df_ncd > 0) {
        const int64_t n = ms->df_ncd * nrhs;
        k_m_absmax<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(
            g->d_M, g->ncoef, ms->ispow, ms->df_c0, ms->df_ncd, nrhs, ms->df_emax);
        ++g->n_launches;
    }
    if (ms->df_nsd > 0) {
        const int64_t n = ms->df_nsd * nrhs;
        k_m_absmax<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(
            g->d_Mp, g->nslotcoef, ms->ispow_slot, ms->df_s0, ms->df_nsd, nrhs, ms->df_emax);
        ++g->n_launches;
    }
    // the coarse levels' multipoles (cells: scaled and unscaled; reaction centres: scaled)
    if (ms->df_ncd > 0) {
        const int64_t n = ms->df_ncd * nrhs;
        k_m_to_df<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(
            g->d_M, g->ncoef, ms->ispow, ms->df_c0, ms->df_ncd, nrhs, ms->df_emax, ms->Mdf, ms->Mudf);
        ++g->n_launches;
    }
    if (ms->df_nsd > 0) {
        const int64_t n = ms->df_nsd * nrhs;
        k_m_to_df<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(
            g->d_Mp, g->nslotcoef, ms->ispow_slot, ms->df_s0, ms->df_nsd, nrhs, ms->df_emax, ms->Mpdf, nullptr);
        ++g->n_launches;
    }
    cuda_check(cudaGetLastError(), "k_m_to_df");
    k_m2l_df<<<dim3(n_items, col_groups(nrhs)), 128, 0, s>>>(g->d_m2l_items, g->d_m2l_ents, g->d_box_level, g->d_p_level, g->d_coef_off,
                                     g->d_slot_of, g->d_slot_coef, ms->ftab_df,
                                     ms->ftab_df + std::max<int64_t>(g->m2lf_len, 1), g->d_m2lf_off, ms->rtab_df,
                                     ms->rtab_rsc, ms->ispow, nrhs, g->ncoef, g->nslotcoef, g->n_m2l_parts, ms->Mdf, ms->Mudf,
                                     ms->df_c0, ms->df_ncd, ms->Mpdf, ms->df_s0, ms->df_nsd, ms->df_emax, g->d_L,
                                     g->d_Lp,
                                     g->d_m2l_part);
    cuda_check(cudaGetLastError(), "k_m2l_df");
    ++g->n_launches;
}

void mixed_m2l(lfmm_geometry_s* g, int nrhs, int min_level, cudaStream_t s) {
    MixedState* ms = g->mixed;
    const TreeHost& t = g->tree;
    if (m2l_tc(g, nrhs, min_level, s)) return;
    const int i0 = g->m2l_item_level_start[min_level];
    const int ni = g->n_m2l_items - i0;
    const int r0 = g->m2l_red_level_start[min_level];
    const int nr = g->m2l_red_level_start[t.D + 1] - r0;
    if (ni > 0) {
        k_m2l32<<<ni, 128, 0, s>>>(g->d_m2l_items + i0, g->d_m2l_ents, g->d_box_level, g->d_p_level, g->d_coef_off,
                                   g->d_slot_of, g->d_slot_coef, ms->ftab, ms->ftab_off, ms->rtab, nrhs, g->ncoef,
                                   g->nslotcoef, g->n_m2l_parts, ms->M, ms->Mp, ms->L, ms->Lp, ms->part);
        cuda_check(cudaGetLastError(), "k_m2l32");
        ++g->n_launches;
    }
    if (nr > 0) {
        k_m2l32_reduce<<<nr, 64, 0, s>>>(g->d_m2l_reds + r0, g->d_box_level, g->d_p_level, g->d_coef_off,
                                         g->d_slot_of, g->d_slot_coef, nrhs, g->ncoef, g->nslotcoef, g->n_m2l_parts,
                                         ms->part, ms->L, ms->Lp);
        cuda_check(cudaGetLastError(), "k_m2l32_reduce");
        ++g->n_launches;
    }
}

}  // namespace lfmm
