// fmm_kernels.cuh -- device kernels of the far field (Sec. 4.1).
//
// One quadtree per layer carries one set of expansions with the layer's
// wavenumber k:
//   multipole  M_n = sum_j Q_j J_n(k rho_j) e^{-i n theta_j}     (about the box centre)
//   local      u(r) = sum_n L_n J_n(k rho) e^{i n theta}         (about the box centre)
// with Q_j = |Gamma_j| Phi_j.  The free-space part uses Graf's addition
// theorem (M2M, M2L with H_{m-n}, L2L).  Every reaction component reuses the
// same multipoles and locals: in the component's image frame (x, h) the
// source-side expansion of the paper, alpha_n = sum Q J_n(k rho) e^{i n theta'}
// (eq. MEcoefficients), is M_n when the height is measured downward
// (theta' = -theta) and (-1)^n M_{-n} when it is measured upward; likewise the
// target-side local expansion (eq. LEformula) lands in L_m or, with (-1)^m, in
// L_{-m}.  The reaction M2L is then the paper's dense translation
// beta_m = sum_n I_{nm} alpha_n (eq. metoleimage) with the moments I_{nm} of
// eq. generalintegral tabulated per box-pair geometry.
#pragma once
#include "devmath.cuh"
#include "sommerfeld.cuh"

namespace lfmm {

#define LFMM_PMAX 80

// P2M over a list of point ranges: entry e expands the points [beg, end) of
// layer lay about (cx, cy) to order p: M_n = sum_j Q_j J_n(k rho_j) e^{-i n theta_j}.
// Used for the leaves (about the cell centres) and for the cells that straddle an
// interface (about their reaction centres).  One CTA (128 threads) per entry.
struct ExpEntry {
    int beg, end, lay, p;
    double cx, cy;
    int64_t off;   // coefficient offset in the output/input array
};

__global__ void k_p2m(const ExpEntry* __restrict__ ent, MediumDev m, const double* __restrict__ px,
                      const double* __restrict__ py, const double* __restrict__ pw, const cd* __restrict__ phi,
                      int64_t n, int nrhs, int64_t stride, cd* __restrict__ M) {
    extern __shared__ double sm[];
    const ExpEntry E = ent[blockIdx.x];
    const int p = E.p, np1 = p + 1;
    double* J = sm;                          // [32][p+1]
    cd* zp = (cd*)(sm + 32 * np1);           // [32][p+1]   z^n, z = e^{-i theta}
    cd* q = zp + 32 * np1;                   // [32] charges of the current column
    const int b0 = E.beg, nb = E.end - E.beg;
    const double k = m.k[E.lay];
    const int nco = 2 * p + 1;
    for (int col = 0; col < nrhs; ++col) {
        // accumulators: thread t owns coefficient indices t, t+128
        cd acc[2] = {mk(0, 0), mk(0, 0)};
        for (int c0 = 0; c0 < nb; c0 += 32) {
            const int cnt = min(32, nb - c0);
            __syncthreads();
            if (threadIdx.x < cnt) {
                const int j = b0 + c0 + threadIdx.x;
                double dx = px[j] - E.cx, dy = py[j] - E.cy;
                double rho = hypot(dx, dy);
                bessel_j_seq(k * rho, p, J + threadIdx.x * np1);
                cd z = (rho > 0.0) ? mk(dx / rho, -dy / rho) : mk(1.0, 0.0);
                cd zz = mk(1.0, 0.0);
                for (int t = 0; t <= p; ++t) { zp[threadIdx.x * np1 + t] = zz; zz = zz * z; }
                q[threadIdx.x] = pw[j] * phi[(int64_t)col * n + j];
            }
            __syncthreads();
            for (int s = 0; s < 2; ++s) {
                int idx = threadIdx.x + 128 * s;
                if (idx >= nco) break;
                int nn = idx - p;
                int an = nn < 0 ? -nn : nn;
                cd a = acc[s];
                for (int j = 0; j < cnt; ++j) {
                    double jv = J[j * np1 + an];
                    cd zn = zp[j * np1 + an];
                    if (nn < 0) { zn = conjc(zn); if (an & 1) jv = -jv; }
                    cfma(a, jv * q[j], zn);
                }
                acc[s] = a;
            }
        }
        for (int s = 0; s < 2; ++s) {
            int idx = threadIdx.x + 128 * s;
            if (idx < nco) M[(int64_t)col * stride + E.off + idx] = acc[s];
        }
    }
}

// M2L into every target box of levels >= l0 (free space and reaction components).
// Work item = (target box, chunk of XT_W output indices); a CTA of 128 threads
// holds XT_W output lanes x 8 slices of the sum over the source index, for
// every list entry of the target in turn, and reduces the slices in a fixed
// order at the end.  Free space (Graf): L_n += sum_m M_m T[m - n].  Reaction
// (eq. generalintegral): beta_m = sum_n I[m][n] alpha_n with the arrival and
// departure index flips; tables are stored column-major (entry (m, n) at
// n (2p+1) + m) so the lanes of a row read consecutive addresses.
__global__ void __launch_bounds__(128) k_m2l(const M2LItem* __restrict__ items, const int* __restrict__ box_level,
                      const int* __restrict__ p_level, const int64_t* __restrict__ coef_off,
                      const int* __restrict__ vf_ptr, const int* __restrict__ vf_src, const int* __restrict__ vf_tab,
                      const cd* __restrict__ m2lf, const int64_t* __restrict__ m2lf_off,
                      const int* __restrict__ vr_ptr, const int* __restrict__ vr_src,
                      const int* __restrict__ vr_key, const int* __restrict__ vr_comp,
                      const int* __restrict__ comp, const ReactKey* __restrict__ rkeys,
                      const cd* __restrict__ m2lr, int nrhs, int64_t ncoef, const cd* __restrict__ Min,
                      cd* __restrict__ Lout, const int* __restrict__ slot_of, const int64_t* __restrict__ slot_coef,
                      int64_t nslotcoef, const cd* __restrict__ Mp, cd* __restrict__ Lp) {
    constexpr int NS = 128 / XT_W;
    __shared__ cd red[3][NS][XT_W];
    const M2LItem it = items[blockIdx.x];
    const int T = it.box;
    const int p = p_level[box_level[T]];
    const int nco = 2 * p + 1;
    const int lane = threadIdx.x % XT_W, sl = threadIdx.x / XT_W;
    const int idx = it.chunk * XT_W + lane;
    const bool live = idx < nco;
    const int nn = idx - p;
    const int tslot[2] = {slot_of[2 * T], slot_of[2 * T + 1]};
    const int f0 = vf_ptr[T], f1 = vf_ptr[T + 1];
    const int r0 = vr_ptr[T], r1 = vr_ptr[T + 1];
    for (int col = 0; col < nrhs; ++col) {
        const cd* Mc = Min + (int64_t)col * ncoef;
        const cd* Mpc = Mp + (int64_t)col * nslotcoef;
        cd acc0 = mk(0, 0), acc1 = mk(0, 0), acc2 = mk(0, 0);   // L, side-0 slot, side-1 slot
        if (live) {
            for (int e = f0; e < f1; ++e) {
                const cd* src = Mc + coef_off[vf_src[e]];
                const cd* tb = m2lf + m2lf_off[vf_tab[e]] + p - nn;   // T[m - n], index (mi - p) - nn + 2p
                for (int mi = sl; mi < nco; mi += NS) cfma(acc0, src[mi], tb[mi]);
            }
            for (int e = r0; e < r1; ++e) {
                const int S = vr_src[e], c = vr_comp[e];
                const int a_dir = comp[4 * c + 1], b_dir = comp[4 * c + 3];
                // source expansion about the reaction centre if S straddles the arrival interface
                const int ssl = slot_of[2 * S + (a_dir == 0 ? 0 : 1)];
                const cd* src = (ssl >= 0) ? (Mpc + slot_coef[ssl]) : (Mc + coef_off[S]);
                // departure down: L_n += beta_n;  departure up: L_{-n} += (-1)^n beta_n
                const int mrow = (b_dir == 1) ? nn : -nn;
                const cd* col_m = m2lr + rkeys[vr_key[e]].off + (mrow + p);
                cd bsum = mk(0, 0);
                if (a_dir == 1) {   // alpha_i = M_i
                    for (int mi = sl; mi < nco; mi += NS) cfma(bsum, col_m[(int64_t)mi * nco], src[mi]);
                } else {            // alpha_i = (-1)^(i-p) M_{2p-i}
                    for (int mi = sl; mi < nco; mi += NS) {
                        cd v = src[2 * p - mi];
                        if ((mi - p) & 1) v = -v;
                        cfma(bsum, col_m[(int64_t)mi * nco], v);
                    }
                }
                if (b_dir == 0 && (mrow & 1)) bsum = -bsum;
                const int side = (b_dir == 0) ? 1 : 0;
                if (tslot[side] < 0) acc0 += bsum;
                else if (side == 0) acc1 += bsum;
                else acc2 += bsum;
            }
        }
        red[0][sl][lane] = acc0;
        red[1][sl][lane] = acc1;
        red[2][sl][lane] = acc2;
        __syncthreads();
        if (live && sl < 3) {
            const int k = sl;
            if (k == 0 || tslot[k - 1] >= 0) {
                cd t = red[k][0][lane];
                for (int q = 1; q < NS; ++q) t += red[k][q][lane];
                if (k == 0) Lout[(int64_t)col * ncoef + coef_off[T] + idx] = t;
                else Lp[(int64_t)col * nslotcoef + slot_coef[tslot[k - 1]] + idx] = t;
            }
        }
        __syncthreads();
    }
}

// L2P over a list of point ranges: y_i += sum_n L_n J_n(k rho_i) e^{i n theta_i}
// about (cx, cy).  Leaves (cell centres) and straddling leaves (reaction centres).
__global__ void k_l2p(const ExpEntry* __restrict__ ent, MediumDev m, const double* __restrict__ px,
                      const double* __restrict__ py, int64_t n, int nrhs, int64_t stride,
                      const cd* __restrict__ L, cd* __restrict__ y) {
    extern __shared__ double sl[];
    const ExpEntry E = ent[blockIdx.x];
    const int p = E.p, np1 = p + 1, nco = 2 * p + 1;
    cd* Ls = (cd*)sl;                               // [nco]
    double* Jall = sl + 2 * nco;                     // [blockDim][p+1]
    const int b0 = E.beg, nb = E.end - E.beg;
    const double k = m.k[E.lay];
    double* J = Jall + threadIdx.x * np1;
    for (int c0 = 0; c0 < nb; c0 += blockDim.x) {
        const int j = b0 + c0 + threadIdx.x;
        const bool act = (c0 + threadIdx.x) < nb;
        cd z = mk(1.0, 0.0);
        if (act) {
            double dx = px[j] - E.cx, dy = py[j] - E.cy;
            double rho = hypot(dx, dy);
            bessel_j_seq(k * rho, p, J);
            if (rho > 0.0) z = mk(dx / rho, dy / rho);
        }
        for (int col = 0; col < nrhs; ++col) {
            __syncthreads();
            for (int i = threadIdx.x; i < nco; i += blockDim.x) Ls[i] = L[(int64_t)col * stride + E.off + i];
            __syncthreads();
            if (act) {
                cd acc = Ls[p] * J[0];
                cd zz = mk(1.0, 0.0);
                for (int t = 1; t <= p; ++t) {
                    zz = zz * z;
                    double jt = J[t];
                    cfma(acc, jt * Ls[p + t], zz);
                    cfma(acc, ((t & 1) ? -jt : jt) * Ls[p - t], conjc(zz));
                }
                y[(int64_t)col * n + j] += acc;
            }
        }
    }
}

// Multipole-to-multipole and local-to-local translations (Graf's addition
// theorem) into the destinations of one level: cell centres and reaction
// centres of straddling cells alike, each with its own list of sources:
//   dst_n (= or +=) sum_j sum_m src_j[m] V_j[n - m + pS_j + pD].
// A CTA of 128 threads owns XT_W consecutive output indices of one
// destination (one per lane of a 16-lane row) and 8 slices of the sum over
// m; the slices are reduced in a fixed order, so results are reproducible.
// Spreading a destination over several CTAs keeps the coarse levels (few
// boxes, orders up to 2p+1 ~ 115) from running on a handful of SMs.
struct XDst {
    int64_t off;          // coefficient offset of the destination
    int p;                // its order
    int in_slots;         // 1: the destination lives in the reaction-centre arrays
    int src_begin, src_end;
};
struct XSrc {
    int64_t off;          // coefficient offset of the source
    int64_t vec_off;      // translation vector V (2 (pS + pD) + 1 entries)
    int p;                // source order
    int in_slots;
};
__global__ void __launch_bounds__(128) k_translate(const XDst* __restrict__ dsts, const XSrc* __restrict__ srcs,
                                                   const cd* __restrict__ vec, int accumulate, int nrhs,
                                                   int64_t ncoef, int64_t nslotcoef, cd* X, cd* Xp) {
    __shared__ cd red[128 / XT_W][XT_W];
    const XDst d = dsts[blockIdx.x];
    const int lane = threadIdx.x % XT_W, sl = threadIdx.x / XT_W;
    const int idx = blockIdx.y * XT_W + lane;
    const int ncD = 2 * d.p + 1;
    for (int col = 0; col < nrhs; ++col) {
        cd a = mk(0, 0);
        if (idx < ncD) {
            for (int j = d.src_begin; j < d.src_end; ++j) {
                const XSrc sr = srcs[j];
                const cd* src = (sr.in_slots ? Xp + (int64_t)col * nslotcoef : X + (int64_t)col * ncoef) + sr.off;
                // V[n - m + hw] with n = idx - pD, m = mi - pS, hw = pS + pD
                const cd* Vb = vec + sr.vec_off + idx + 2 * sr.p;
                const int ncS = 2 * sr.p + 1;
                for (int mi = sl; mi < ncS; mi += 128 / XT_W) cfma(a, src[mi], Vb[-mi]);
            }
        }
        red[sl][lane] = a;
        __syncthreads();
        if (sl == 0 && idx < ncD) {
            cd t = red[0][lane];
            for (int q = 1; q < 128 / XT_W; ++q) t += red[q][lane];
            cd* dst = (d.in_slots ? Xp + (int64_t)col * nslotcoef : X + (int64_t)col * ncoef) + d.off + idx;
            if (accumulate) *dst += t;
            else *dst = t;
        }
        __syncthreads();
    }
}

// Reaction M2L moment tables (eq. generalintegral): one CTA per (key, 32x32 tile).
struct TableWork {
    int key;
    int m0, n0;   // first row / column of the tile (indices from -p)
};

__global__ void __launch_bounds__(256) k_react_tables(MediumDev med, QuadRule q, const ReactKey* __restrict__ keys,
                                                      const TableWork* __restrict__ work,
                                                      const int* __restrict__ comp, cd* __restrict__ out) {
    extern __shared__ cd st[];
    const TableWork wk = work[blockIdx.x];
    const ReactKey K = keys[wk.key];
    const int c = K.comp;
    const int ls = comp[4 * c], a = comp[4 * c + 1], lt = comp[4 * c + 2], b = comp[4 * c + 3];
    const int pS = K.pS, pT = K.pT;
    const int ncS = 2 * pS + 1, ncT = 2 * pT + 1;
    const double ka = med.k[ls], kb = med.k[lt];
    // smem layout for a chunk of CH nodes
    const int CH = 16;
    cd* Up = st;                       // [CH][32]  u^n  for the tile's n
    cd* Um = Up + CH * 32;             // [CH][32]  u^-n
    cd* Vp = Um + CH * 32;             // [CH][32]  v^-m for the tile's m
    cd* Vm = Vp + CH * 32;             // [CH][32]  v^m
    cd* Fp = Vm + CH * 32;             // [CH]
    cd* Fm = Fp + CH;                  // [CH]
    cd* uu = Fm + CH;                  // [CH] u
    cd* vv = uu + CH;                  // [CH] v
    // table rule: finer detour (panels grow with the orders) and finer rays
    QuadRule qt = q;
    qt.es_v0 = q.tab_es_v0;
    qt.es_hv = q.tab_es_hv;
    qt.nes = q.tab_nes;
    double h;
    const int P = detour_panels(q, K.X, K.D, &h) * q.tab_panel_mult + (pS + pT);
    const int ntot = P * 8 + 2 * qt.nes;
    const int tm = threadIdx.x >> 3;          // 0..31 row within tile
    const int tn = (threadIdx.x & 7) * 4;     // 0..28 first column within tile
    cd acc[4] = {mk(0, 0), mk(0, 0), mk(0, 0), mk(0, 0)};
    for (int j0 = 0; j0 < ntot; j0 += CH) {
        const int cnt = min(CH, ntot - j0);
        __syncthreads();
        if (threadIdx.x < cnt) {
            QuadNode nd = contour_node(qt, j0 + threadIdx.x, P, h, K.X, K.D);
            cd S = sigma_comp(med, nd.lam, ls, a, lt, b);
            cd kya = ky_of(ka, nd.lam), kyb = ky_of(kb, nd.lam);
            cd E = eikh(kya, K.hS) * eikh(kyb, K.hT);
            cd SE = S * E;
            Fp[threadIdx.x] = SE * nd.fp;
            Fm[threadIdx.x] = SE * nd.fm;
            uu[threadIdx.x] = w_of(kya, nd.lam, ka);
            vv[threadIdx.x] = w_of(kyb, nd.lam, kb);
        }
        __syncthreads();
        // power tables: thread (node r, slot s) for 16 x 32 entries, 2 passes
        for (int e = threadIdx.x; e < cnt * 32; e += blockDim.x) {
            int r = e >> 5, s = e & 31;
            int nn = wk.n0 + s, mm = wk.m0 + s;
            cd u = uu[r], v = vv[r];
            cd ui = cinv(u), vi = cinv(v);
            // integer powers by binary exponentiation
            auto ipow = [](cd base, int e2) {
                cd r2 = mk(1.0, 0.0);
                cd bb = base;
                while (e2 > 0) { if (e2 & 1) r2 = r2 * bb; bb = bb * bb; e2 >>= 1; }
                return r2;
            };
            Up[r * 32 + s] = (nn >= 0) ? ipow(u, nn) : ipow(ui, -nn);
            Um[r * 32 + s] = (nn >= 0) ? ipow(ui, nn) : ipow(u, -nn);
            Vp[r * 32 + s] = (mm >= 0) ? ipow(vi, mm) : ipow(v, -mm);
            Vm[r * 32 + s] = (mm >= 0) ? ipow(v, mm) : ipow(vi, -mm);
        }
        __syncthreads();
        for (int r = 0; r < cnt; ++r) {
            cd a1 = Fp[r] * Vp[r * 32 + tm];
            cd a2 = Fm[r] * Vm[r * 32 + tm];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                cfma(acc[t], a1, Up[r * 32 + tn + t]);
                cfma(acc[t], a2, Um[r * 32 + tn + t]);
            }
        }
    }
    const int mm = wk.m0 + tm;
    if (mm <= pT) {
        for (int t = 0; t < 4; ++t) {
            int nn = wk.n0 + tn + t;
            if (nn <= pS) out[K.off + (int64_t)(nn + pS) * ncT + (mm + pT)] = acc[t];
        }
    }
}

}  // namespace lfmm
