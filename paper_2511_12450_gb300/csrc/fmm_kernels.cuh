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
#include <algorithm>

#include "devmath.cuh"
#include "sommerfeld.cuh"

namespace lfmm {

#define LFMM_PMAX 80

// P2M over a list of point ranges: entry e expands the points [beg, end) of
// layer lay about (cx, cy) to order p: M_n = sum_j Q_j J_n(k rho_j) e^{-i n theta_j}.
// Used for the leaves (about the cell centres) and for the cells that straddle an
// interface (about their reaction centres).  One CTA (128 threads) per entry.

// Consecutive expansion entries whose points are processed by one CTA together
// (at most EXP_GROUP_PTS points, or a single larger entry).

// Point t of a group: its entry (relative index) and point index.
__device__ __forceinline__ void group_point(const ExpEntry* __restrict__ ent, int e0, int e1, int t, int* er, int* j) {
    int e = e0, base = 0;
    while (e + 1 < e1 && t >= base + (ent[e].end - ent[e].beg)) { base += ent[e].end - ent[e].beg; ++e; }
    *er = e - e0;
    *j = ent[e].beg + (t - base);
}

// P2M about the entries' centres (leaves about cell centres, straddling leaves
// about their reaction centres): M_n = sum_j q_j J_n(k rho_j) e^{-i n theta_j},
// q_j = |Gamma_j| phi_j.  Phase 1, one thread per point of the group: its basis
// row u_{j,n} = J_n(k rho_j) e^{-i n theta_j} for n = -p..p (J_{-n} = (-1)^n J_n,
// e^{+i n theta} = conj) into shared memory.  Phase 2, one thread per (entry,
// coefficient): the sum over the entry's points, pure complex FMAs.
// Combined field (normals given): the row is the basis of a dipole along n_j
// plus -i k times the charge's, E_n = n_j . grad u_n - i k u_n, with
// n . grad u_n = (k/2)(conj(nu) u_{n-1} - nu u_{n+1}), nu = n_x + i n_y (from
// (d_x +- i d_y) J_m e^{i m theta} = -+k J_{m+-1} e^{i (m+-1) theta}); the
// translations are linear and carry it unchanged.
__device__ __forceinline__ void p2m_group(int gi, const ExpGroup* __restrict__ groups,
                                          const ExpEntry* __restrict__ ent, const MediumDev& m,
                                          const double* __restrict__ pw, const double* __restrict__ nx,
                                          const double* __restrict__ ny, const cd* __restrict__ basis,
                                          int bstride, const cd* __restrict__ phi, int64_t n,
                                          int nrhs, int64_t stride, cd* __restrict__ M) {
    extern __shared__ cd su[];   // [npts][rs] basis rows, then [npts] q, then [nent + 1] point offsets (ints)
    const ExpGroup G = groups[gi];
    const int p = ent[G.e0].p, nco = 2 * p + 1;
    const bool cf = nx != nullptr;
    const int pb = cf ? p + 1 : p, rs = 2 * pb + 1;   // order and length of the plain basis rows
    const int ne = G.e1 - G.e0;
    cd* sq = su + (size_t)G.npts * rs;
    int* soff = (int*)(sq + G.npts);
    if (threadIdx.x == 0) {
        int o = 0;
        for (int e = 0; e < ne; ++e) { soff[e] = o; o += ent[G.e0 + e].end - ent[G.e0 + e].beg; }
        soff[ne] = o;
    }
    for (int t = threadIdx.x; t < G.npts; t += blockDim.x) {
        int er, j;
        group_point(ent, G.e0, G.e1, t, &er, &j);
        const ExpEntry& E = ent[G.e0 + er];
        cd* u = su + (size_t)t * rs;
        // u_n = J_n(k rho) e^{-i n theta} = conj of the stored basis, n = 0..pb, into slots pb..2pb
        const cd* b = basis + (E.brow + (j - E.beg)) * (int64_t)bstride;
        for (int k2 = 0; k2 <= pb; ++k2) {
            const cd v = b[k2];
            u[pb + k2] = mk(v.x, -v.y);
        }
        // u_{-n} = (-1)^n conj(u_n) into slots pb-1..0; the signs by integer bit flips
        // (no FP64 instruction)
        for (int k2 = 1; k2 <= pb; ++k2) {
            const cd v = u[pb + k2];
            u[pb - k2] = mk(dsign(v.x, k2), dsign(v.y, k2 + 1));
        }
        if (cf) {   // E_n into slot n + p from u_{n-1}, u_n, u_{n+1} (slots n+p, n+p+1, n+p+2);
                    // ascending n overwrites only u_{n-1}, which later n do not read
            const double k = m.k[E.lay];
            const cd nu = mk(nx[j], ny[j]), nub = conjc(nu);
            for (int s2 = 0; s2 < nco; ++s2) {
                const cd um = u[s2], u0 = u[s2 + 1], up = u[s2 + 2];
                const cd d = 0.5 * (nub * um - nu * up);
                u[s2] = k * mk(d.x + u0.y, d.y - u0.x);   // k (d - i u_n)
            }
        }
    }
    for (int col = 0; col < nrhs; ++col) {
        __syncthreads();
        for (int t = threadIdx.x; t < G.npts; t += blockDim.x) {
            int er, j;
            group_point(ent, G.e0, G.e1, t, &er, &j);
            sq[t] = pw[j] * phi[(int64_t)col * n + j];
        }
        __syncthreads();
        for (int task = threadIdx.x; task < ne * nco; task += blockDim.x) {
            const int er = task / nco, idx = task - er * nco;
            cd a = mk(0, 0);
            for (int t = soff[er]; t < soff[er + 1]; ++t) cfma(a, sq[t], su[(size_t)t * rs + idx]);
            M[(int64_t)col * stride + ent[G.e0 + er].off + idx] = a;
        }
    }
}
__global__ void __launch_bounds__(128) k_p2m(const ExpGroup* __restrict__ groups, const ExpEntry* __restrict__ ent,
                      MediumDev m, const double* __restrict__ pw, const double* __restrict__ nx,
                      const double* __restrict__ ny, const cd* __restrict__ basis, int bstride,
                      const cd* __restrict__ phi, int64_t n, int nrhs, int64_t stride, cd* __restrict__ M) {
    p2m_group(blockIdx.x, groups, ent, m, pw, nx, ny, basis, bstride, phi, n, nrhs, stride, M);
}

// The expansion basis of every (entry, point), computed once per geometry:
// b_n = J_n(k rho) e^{i n theta}, n = 0..ord, with (rho, theta) the point's polar
// coordinates about the entry's centre (the cell centre, or a straddling leaf's reaction
// centre).  L2P uses b_n, P2M its conjugate.  e^{i n theta} by powers upward from 1.
__global__ void __launch_bounds__(128) k_basis(const ExpGroup* __restrict__ groups, const ExpEntry* __restrict__ ent,
                                               MediumDev m, const double* __restrict__ px,
                                               const double* __restrict__ py, int ord, cd* __restrict__ basis) {
    extern __shared__ double sjb[];   // [npts][ord + 1] J_n
    const ExpGroup G = groups[blockIdx.x];
    for (int t = threadIdx.x; t < G.npts; t += blockDim.x) {
        int er, j;
        group_point(ent, G.e0, G.e1, t, &er, &j);
        const ExpEntry& E = ent[G.e0 + er];
        const double dx = px[j] - E.cx, dy = py[j] - E.cy;
        const double rho = hypot(dx, dy);
        double* J = sjb + (size_t)t * (ord + 1);
        bessel_j_seq_small(m.k[E.lay] * rho, ord, J);
        const double irho = (rho > 0.0) ? 1.0 / rho : 0.0;
        const cd z = (rho > 0.0) ? mk(dx * irho, dy * irho) : mk(1.0, 0.0);
        cd* b = basis + (E.brow + (j - E.beg)) * (int64_t)(ord + 1);
        b[0] = mk(J[0], 0.0);
        cd zz = mk(1.0, 0.0);
        for (int k2 = 1; k2 <= ord; ++k2) {
            zz = zz * z;
            b[k2] = mk(J[k2] * zz.x, J[k2] * zz.y);
        }
    }
}

// M2L into the target boxes of levels >= l0 (free space and reaction components).
// A CTA of 128 threads takes one work item: W output lanes (W = XT_W, or every
// coefficient, see lane_width) x 128 / W slices of the sum over the source
// index, over the item's range of list entries, whose descriptors are staged in
// shared memory 64 at a time; the slices are reduced
// in a fixed order at the end.  Free space (Graf): L_n += sum_m M_m T[m - n]
// (Toeplitz vector per table).  Reaction (eq. generalintegral): beta_m =
// sum_n I[m][n] alpha_n with the arrival and departure index flips; moment
// tables are column-major (entry (m, n) at n (2p+1) + m).
#define M2L_STAGE 64

__device__ __forceinline__ void m2l_item(int ii, const M2LItem* __restrict__ items, const M2LEnt* __restrict__ ents,
                      const int* __restrict__ box_level, const int* __restrict__ p_level,
                      const int64_t* __restrict__ coef_off, const int* __restrict__ slot_of,
                      const int64_t* __restrict__ slot_coef, const cd* __restrict__ m2lf,
                      const int64_t* __restrict__ m2lf_off, const cd* __restrict__ m2lr, int nrhs, int64_t ncoef,
                      int64_t nslotcoef, int nparts, const cd* __restrict__ Min, const cd* __restrict__ Mp,
                      cd* __restrict__ Lout, cd* __restrict__ Lp, cd* __restrict__ part) {
    __shared__ cd red[3 * 128];
    __shared__ M2LEnt se[M2L_STAGE];
    const M2LItem it = items[ii];
    const int T = it.box;
    const int p = p_level[box_level[T]];
    const int nco = 2 * p + 1;
    const int W = it.w, NS = 128 / W;
    const int lane = threadIdx.x % W, sl = threadIdx.x / W;
    const int idx = it.chunk * W + lane;
    const bool live = sl < NS && idx < nco;
    const int nn = idx - p;
    for (int col = 0; col < nrhs; ++col) {
        const cd* Mc = Min + (int64_t)col * ncoef;
        const cd* Mpc = Mp + (int64_t)col * nslotcoef;
        cd acc0 = mk(0, 0), acc1 = mk(0, 0), acc2 = mk(0, 0);   // L, side-0 / side-1 reaction centre
        for (int eb = it.e0; eb < it.e1; eb += M2L_STAGE) {
            const int cnt = min(M2L_STAGE, it.e1 - eb);
            __syncthreads();
            if (threadIdx.x < cnt) se[threadIdx.x] = ents[eb + threadIdx.x];
            __syncthreads();
            if (!live) continue;
            for (int q = 0; q < cnt; ++q) {
                const M2LEnt E = se[q];
                if (!(E.flags & M2L_REACT)) {
                    const cd* src = Mc + E.src;
                    const cd* tb = m2lf + m2lf_off[E.tab] + p - nn;   // T[m - n] at (mi - p) - nn + 2p
                    for (int mi = sl; mi < nco; mi += NS) cfma(acc0, src[mi], tb[mi]);
                } else {
                    const cd* src = ((E.flags & M2L_SRC_SLOT) ? Mpc : Mc) + E.src;
                    const bool bdown = (E.flags & M2L_B_DOWN) != 0;
                    // departure down: L_n += beta_n;  departure up: L_{-n} += (-1)^n beta_n
                    const int mrow = bdown ? nn : -nn;
                    // column of row mrow; a mirrored table is read at (-mrow, -n)
                    const bool flip = (E.flags & M2L_FLIP) != 0;
                    const cd* col_m = m2lr + E.tab + (flip ? (p - mrow) + (int64_t)2 * p * nco : (mrow + p));
                    const int64_t cs = flip ? -(int64_t)nco : (int64_t)nco;
                    cd bsum = mk(0, 0);
                    if (E.flags & M2L_A_DOWN) {   // alpha_i = M_i
                        for (int mi = sl; mi < nco; mi += NS) cfma(bsum, col_m[mi * cs], src[mi]);
                    } else {                      // alpha_i = (-1)^(i-p) M_{2p-i}
                        for (int mi = sl; mi < nco; mi += NS) cfma(bsum, col_m[mi * cs], csign(src[2 * p - mi], mi - p));
                    }
                    bsum = csign(bsum, (!bdown) & mrow);
                    const int dst = (E.flags >> M2L_DST_SHIFT) & 3;
                    if (dst == 0) acc0 += bsum;
                    else if (dst == 1) acc1 += bsum;
                    else acc2 += bsum;
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
            cd t = red[(k * NS) * W + ln];
            for (int q = 1; q < NS; ++q) t += red[(k * NS + q) * W + ln];
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
__global__ void __launch_bounds__(128) k_m2l(const M2LItem* __restrict__ items, const M2LEnt* __restrict__ ents,
                      const int* __restrict__ box_level, const int* __restrict__ p_level,
                      const int64_t* __restrict__ coef_off, const int* __restrict__ slot_of,
                      const int64_t* __restrict__ slot_coef, const cd* __restrict__ m2lf,
                      const int64_t* __restrict__ m2lf_off, const cd* __restrict__ m2lr, int nrhs, int64_t ncoef,
                      int64_t nslotcoef, int nparts, const cd* __restrict__ Min, const cd* __restrict__ Mp,
                      cd* __restrict__ Lout, cd* __restrict__ Lp, cd* __restrict__ part) {
    m2l_item(blockIdx.x, items, ents, box_level, p_level, coef_off, slot_of, slot_coef, m2lf, m2lf_off, m2lr, nrhs,
             ncoef, nslotcoef, nparts, Min, Mp, Lout, Lp, part);
}
// Sum the partial results of split (box, chunk)s in part order and write them.
__device__ __forceinline__ void m2l_reduce_one(int ri, const M2LReduce* __restrict__ reds,
                      const int* __restrict__ box_level, const int* __restrict__ p_level,
                      const int64_t* __restrict__ coef_off, const int* __restrict__ slot_of,
                      const int64_t* __restrict__ slot_coef, int nrhs, int64_t ncoef, int64_t nslotcoef, int nparts,
                      const cd* __restrict__ part, cd* __restrict__ Lout, cd* __restrict__ Lp) {
    const M2LReduce r = reds[ri];
    const int p = p_level[box_level[r.box]];
    const int lane = threadIdx.x % XT_W, k = threadIdx.x / XT_W;   // k < 4; 3 used
    const int idx = r.chunk * XT_W + lane;
    if (k >= 3 || idx >= 2 * p + 1) return;
    const int ts = (k == 0) ? -1 : slot_of[2 * r.box + k - 1];
    if (k > 0 && ts < 0) return;
    for (int col = 0; col < nrhs; ++col) {
        cd t = mk(0, 0);
        for (int q = 0; q < r.nparts; ++q) t += part[(((int64_t)col * nparts + r.part0 + q) * 3 + k) * XT_W + lane];
        if (k == 0) Lout[(int64_t)col * ncoef + coef_off[r.box] + idx] = t;
        else Lp[(int64_t)col * nslotcoef + slot_coef[ts] + idx] = t;
    }
}
__global__ void __launch_bounds__(64) k_m2l_reduce(const M2LReduce* __restrict__ reds,
                      const int* __restrict__ box_level, const int* __restrict__ p_level,
                      const int64_t* __restrict__ coef_off, const int* __restrict__ slot_of,
                      const int64_t* __restrict__ slot_coef, int nrhs, int64_t ncoef, int64_t nslotcoef, int nparts,
                      const cd* __restrict__ part, cd* __restrict__ Lout, cd* __restrict__ Lp) {
    m2l_reduce_one(blockIdx.x, reds, box_level, p_level, coef_off, slot_of, slot_coef, nrhs, ncoef, nslotcoef, nparts,
                   part, Lout, Lp);
}

// L2P over a list of point ranges: y_i += sum_n L_n J_n(k rho_i) e^{i n theta_i}
// about (cx, cy).  Leaves (cell centres) and straddling leaves (reaction centres).
__device__ __forceinline__ void l2p_group(int gi, const ExpGroup* __restrict__ groups,
                      const ExpEntry* __restrict__ ent, const cd* __restrict__ basis, int bstride, int64_t n,
                      int nrhs, int64_t stride, const cd* __restrict__ L, cd* __restrict__ y) {
    // y_j += sum_n L_n J_n(k rho_j) e^{i n theta_j}.  Per entry, A_n = L_n and
    // B_n = (-1)^n L_{-n} are folded into P_n = A_n + B_n and Q_n = A_n - B_n, so
    // that A_n z^n + B_n conj(z^n) = P_n cos(n theta) + i Q_n sin(n theta); the point's
    // J_n cos(n theta) and J_n sin(n theta) are its stored basis row.
    extern __shared__ cd sPQ[];   // [nent][2][p+1] (P, Q)
    const ExpGroup G = groups[gi];
    const int p = ent[G.e0].p, np1 = p + 1;
    const int ne = G.e1 - G.e0;
    for (int col = 0; col < nrhs; ++col) {
        __syncthreads();
        for (int i = threadIdx.x; i < ne * np1; i += blockDim.x) {
            const int er = i / np1, k2 = i - er * np1;
            const cd* Le = L + (int64_t)col * stride + ent[G.e0 + er].off;
            const cd A = Le[p + k2];
            const cd B = csign(Le[p - k2], k2);
            if (k2 == 0) { sPQ[(er * 2) * np1] = A; sPQ[(er * 2 + 1) * np1] = mk(0, 0); }
            else { sPQ[(er * 2) * np1 + k2] = A + B; sPQ[(er * 2 + 1) * np1 + k2] = A - B; }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < G.npts; t += blockDim.x) {
            int er, j;
            group_point(ent, G.e0, G.e1, t, &er, &j);
            const ExpEntry& E = ent[G.e0 + er];
            const cd* b = basis + (E.brow + (j - E.beg)) * (int64_t)bstride;
            const cd* P = sPQ + (er * 2) * np1;
            const cd* Q = P + np1;
            cd acc = P[0] * b[0].x;
            for (int k2 = 1; k2 <= p; ++k2) {
                const cd v = b[k2];
                acc.x = fma(P[k2].x, v.x, fma(-Q[k2].y, v.y, acc.x));
                acc.y = fma(P[k2].y, v.x, fma(Q[k2].x, v.y, acc.y));
            }
            y[(int64_t)col * n + j] += acc;
        }
    }
}
__global__ void __launch_bounds__(128) k_l2p(const ExpGroup* __restrict__ groups, const ExpEntry* __restrict__ ent,
                      const cd* __restrict__ basis, int bstride, int64_t n, int nrhs, int64_t stride,
                      const cd* __restrict__ L, cd* __restrict__ y) {
    l2p_group(blockIdx.x, groups, ent, basis, bstride, n, nrhs, stride, L, y);
}

// Multipole-to-multipole and local-to-local translations (Graf's addition theorem),
// one launch per level and pass over two kinds of work:
//  - families (QuadX): a parent cell and its children about cell centres.  The
//    children's offsets d_q = (+-w/2, +-w/2) share one length, and their angles are
//    quarter turns apart, so child q's vector is the quadrant-3 (base) vector times a
//    phase: V^q_k = B_k om_q^k, om_q a power of -i (M2M; L2L uses the conjugates).  With
//    s = (n - m) mod 4 (M2M) or (m - n) mod 4 (L2L),
//      M2M:  M^P_n = sum_s sum_{m: s} B_{n-m} S^s_m,   S^s_m = sum_q om_q^s M^q_m,
//      L2L:  L^q_n = sum_s conj(om_q)^s T^s_n,        T^s_n = sum_{m: s} C_{m-n} L^P_m,
//    where S and the sum over s are 4-point transforms (additions, negations and
//    exchanges of real and imaginary parts).  A family thus costs one Toeplitz
//    product instead of one per child.  The work is by warps: lane (n, s) of a round
//    (32 consecutive pairs, 8 outputs x 4 residues) sums the terms of residue s of
//    output n, and the 4 lanes of an output combine by shuffles in a fixed order.
//    Each warp first stages its base vector and sources in shared memory;
//  - reaction centres of straddling cells, and the cells that take a straddling
//    parent's reaction-centre local (XDst), one CTA each, a sum over their own sources,
//      dst_n (= or +=) sum_j sum_m src_j[m] V_j[n - m + pS_j + pD].
//    A CTA of 128 threads owns w consecutive output indices (one per lane of a w-lane
//    row; w = XT_W or all 2p+1 of them, see lane_width) and 128 / w slices of the sum
//    over m, reduced in a fixed order; each source and its vector window are staged in
//    shared memory.
// Every sum runs in a fixed order, so results are reproducible.
struct XPass {
    const XDst* dsts;
    const XSrc* srcs;
    const cd* vec;
    const QuadX* qx;
    int nq, nd, nch, w;   // families, reaction-centre destinations, chunks of w outputs per destination
    int fch, fr;          // warps per family, rounds of 32 (n, s) pairs per warp
    int pS, pD;           // the families' source and destination orders
    int down, accumulate; // L2L; add into the destinations (M2M always writes)
    int64_t ncoef, nslotcoef;
    cd *X, *Xp;
};
// dynamic shared memory of a pass (complex values): per family warp (4 per CTA) its base
// vector and (M2M) the 4 transformed source vectors or (L2L) the parent's local; per
// reaction-centre CTA the 128 partial sums, one source and the window of its vector
inline size_t xpass_smem(int down, int pS, int pD, int w) {
    const int ncS = 2 * pS + 1, nv = 2 * (pS + pD) + 1;
    const int fam = 4 * ((down ? ncS : 4 * ncS) + nv);
    const int dst = 128 + ncS + w + 2 * pS;
    return sizeof(cd) * (size_t)std::max(fam, dst);
}

__device__ __forceinline__ void translate_dst(int di, int chunk, const XPass& P, int col0, int col1, cd* sm) {
    const XDst d = P.dsts[di];
    const int w = P.w, ns = 128 / w;
    const int lane = threadIdx.x % w, sl = threadIdx.x / w;
    const int idx = chunk * w + lane;
    const int ncD = 2 * d.p + 1, ncS = 2 * P.pS + 1;   // every source of a pass has the order pS
    const bool live = sl < ns && idx < ncD;
    cd* red = sm;
    cd* xs = sm + 128;          // the source
    cd* vs = xs + ncS;          // V[chunk w .. chunk w + w - 1 + 2 pS] (n - m + hw over this chunk)
    const int nv = w + 2 * P.pS;
    for (int col = col0; col < col1; ++col) {
        cd a = mk(0, 0);
        for (int j = d.src_begin; j < d.src_end; ++j) {
            const XSrc sr = P.srcs[j];
            const cd* src = (sr.in_slots ? P.Xp + (int64_t)col * P.nslotcoef : P.X + (int64_t)col * P.ncoef) + sr.off;
            const cd* V = P.vec + sr.vec_off + chunk * w;
            const int nvv = min(nv, 2 * (P.pS + d.p) + 1 - chunk * w);   // the vector's end
            __syncthreads();
            for (int i = threadIdx.x; i < ncS; i += blockDim.x) xs[i] = src[i];
            for (int i = threadIdx.x; i < nvv; i += blockDim.x) vs[i] = V[i];
            __syncthreads();
            // V[n - m + hw] with n = idx - pD, m = mi - pS, hw = pS + pD: vs[lane + 2 pS - mi]
            if (live)
                for (int mi = sl; mi < ncS; mi += ns) cfma(a, xs[mi], vs[lane + 2 * P.pS - mi]);
        }
        if (sl < ns) red[sl * w + lane] = a;
        __syncthreads();
        if (sl == 0 && idx < ncD) {
            cd t = red[lane];
            for (int q = 1; q < ns; ++q) t += red[q * w + lane];
            cd* dst = (d.in_slots ? P.Xp + (int64_t)col * P.nslotcoef : P.X + (int64_t)col * P.ncoef) + d.off + idx;
            if (P.accumulate) *dst += t;
            else *dst = t;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ cd mul_i(cd v) { return mk(-v.y, v.x); }   // i v
__device__ __forceinline__ cd shfl_xor_cd(cd v, int m) {
    return mk(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
// sum over the 4 lanes of an output, the same value and order in each
__device__ __forceinline__ cd quad_lane_sum(cd a) {
    a += shfl_xor_cd(a, 1);
    return a + shfl_xor_cd(a, 2);
}

// M2M of one family, warp part `chunk`: the parent's multipole from its children's.
// S: this warp's 4 (2 pS + 1) shared values.  Each lane runs two rounds at once
// (outputs ni and ni + 8, the same residue class of m).
__device__ __forceinline__ void fam_up(int fam, int chunk, const XPass& P, int col0, int col1, cd* S) {
    const QuadX f = P.qx[fam];
    const int lane = threadIdx.x & 31, s = lane & 3;
    const int ncS = 2 * P.pS + 1, ncD = 2 * P.pD + 1, nv = 2 * (P.pS + P.pD) + 1;
    const cd z = mk(0, 0);
    cd* Bs = S + 4 * ncS;   // the base vector
    for (int i = lane; i < nv; i += 32) Bs[i] = P.vec[f.vup + i];
    for (int col = col0; col < col1; ++col) {
        const cd* Xc = P.X + (int64_t)col * P.ncoef;
        __syncwarp();
        for (int mi = lane; mi < ncS; mi += 32) {
            // om_q = 1, -i, -1, i for the quadrants 3, 2, 0, 1
            const cd m0 = f.ch[0] >= 0 ? Xc[f.ch[0] + mi] : z, m1 = f.ch[1] >= 0 ? Xc[f.ch[1] + mi] : z;
            const cd m2 = f.ch[2] >= 0 ? Xc[f.ch[2] + mi] : z, m3 = f.ch[3] >= 0 ? Xc[f.ch[3] + mi] : z;
            const cd u = m3 + m0, v = m2 + m1, x = m3 - m0, iy = mul_i(m2 - m1);
            S[mi] = u + v;
            S[ncS + mi] = x - iy;
            S[2 * ncS + mi] = u - v;
            S[3 * ncS + mi] = x + iy;
        }
        __syncwarp();
        const cd* Ss = S + s * ncS;
        for (int k = 0; k < P.fr; k += 2) {
            const int ni = (((chunk * P.fr + k) << 5) + lane) >> 2;   // output index; ni + 8 in round k + 1
            const bool two = k + 1 < P.fr;
            cd a = z, a2 = z;
            if (ni < ncD) {
                // (n - m) = (ni - pD) - (mi - pS) = s (mod 4); B[n - m + hw] = Vb[-mi]
                const cd* Vb = Bs + ni + 2 * P.pS;
                const int mi0 = (ni - P.pD + P.pS - s) & 3;
                if (two) {
                    // past the last output the second sum reads the last one's terms (not stored),
                    // so every lane runs the same loop
                    const cd* Vb2 = Vb + min(8, ncD - 1 - ni);
                    for (int mi = mi0; mi < ncS; mi += 4) {
                        const cd sv = Ss[mi];
                        cfma(a, sv, Vb[-mi]);
                        cfma(a2, sv, Vb2[-mi]);
                    }
                } else {
                    for (int mi = mi0; mi < ncS; mi += 4) cfma(a, Ss[mi], Vb[-mi]);
                }
            }
            a = quad_lane_sum(a);
            if (s == 0 && ni < ncD) P.X[(int64_t)col * P.ncoef + f.par + ni] = a;
            if (two) {
                a2 = quad_lane_sum(a2);
                if (s == 0 && ni + 8 < ncD) P.X[(int64_t)col * P.ncoef + f.par + ni + 8] = a2;
            }
        }
    }
}

// lane s's child after the L2L transform (quadrant 3, 0, 2, 1 for s = 0, 1, 2, 3): from
// the residue sums T_s of one output, conj(om_q) = 1, i, -1, -i for the quadrants
// 3, 2, 0, 1:  e = T0 + T2, g = T1 + T3, h = T0 - T2, k = T1 - T3, then
// q3 = e + g, q0 = e - g, q2 = h + i k, q1 = h - i k
__device__ __forceinline__ cd quad_lane_transform(cd a, int s) {
    const cd o2 = shfl_xor_cd(a, 2);
    const cd b = (s < 2) ? a + o2 : o2 - a;
    const cd o1 = shfl_xor_cd(b, 1);
    return (s == 0) ? b + o1 : (s == 1) ? o1 - b : (s == 2) ? b + mul_i(o1) : o1 - mul_i(b);
}

// L2L of one family, warp part `chunk`: the children's locals from the parent's (the
// children in dn_skip are destinations of their own)
// Sm: this warp's shared values, the parent's local then the base vector
__device__ __forceinline__ void fam_dn(int fam, int chunk, const XPass& P, int col0, int col1, cd* Sm) {
    const QuadX f = P.qx[fam];
    const int lane = threadIdx.x & 31, s = lane & 3;
    const int ncS = 2 * P.pS + 1, ncD = 2 * P.pD + 1, nv = 2 * (P.pS + P.pD) + 1;
    const int q = (0x1203 >> (4 * s)) & 15;   // the child lane s holds after the transform
    const int64_t chq = ((f.dn_skip >> q) & 1) ? -1 : P.qx[fam].ch[q];
    const cd z = mk(0, 0);
    cd* src = Sm;
    cd* Cs = Sm + ncS;
    for (int i = lane; i < nv; i += 32) Cs[i] = P.vec[f.vdn + i];
    for (int col = col0; col < col1; ++col) {
        const cd* Lp = P.X + (int64_t)col * P.ncoef + f.par;
        __syncwarp();
        for (int i = lane; i < ncS; i += 32) src[i] = Lp[i];
        __syncwarp();
        cd* Xc = P.X + (int64_t)col * P.ncoef + chq;
        for (int k = 0; k < P.fr; k += 2) {
            const int ni = (((chunk * P.fr + k) << 5) + lane) >> 2;
            const bool two = k + 1 < P.fr;
            cd a = z, a2 = z;
            if (ni < ncD) {
                // (m - n) = (mi - pS) - (ni - pD) = s (mod 4); C_{m-n} = Vb[-mi]
                const cd* Vb = Cs + ni + 2 * P.pS;
                const int mi0 = (ni - P.pD + P.pS + s) & 3;
                if (two) {
                    const cd* Vb2 = Vb + min(8, ncD - 1 - ni);   // as fam_up
                    for (int mi = mi0; mi < ncS; mi += 4) {
                        const cd sv = src[mi];
                        cfma(a, sv, Vb[-mi]);
                        cfma(a2, sv, Vb2[-mi]);
                    }
                } else {
                    for (int mi = mi0; mi < ncS; mi += 4) cfma(a, src[mi], Vb[-mi]);
                }
            }
            const cd out = quad_lane_transform(a, s);
            if (ni < ncD && chq >= 0) {
                if (P.accumulate) Xc[ni] += out;
                else Xc[ni] = out;
            }
            if (two) {
                const cd out2 = quad_lane_transform(a2, s);
                if (ni + 8 < ncD && chq >= 0) {
                    if (P.accumulate) Xc[ni + 8] += out2;
                    else Xc[ni + 8] = out2;
                }
            }
        }
    }
}

// CTA b of a pass: family warps first (4 per CTA), then reaction-centre destinations
__device__ __forceinline__ void translate_item(int b, const XPass& P, int col0, int col1, cd* sm) {
    const int fb = xpass_fam_ctas(P.nq, P.fch);
    if (b < fb) {
        const int gw = b * 4 + (threadIdx.x >> 5);
        if (gw >= P.nq * P.fch) return;   // whole warps; the family work has no CTA barrier
        const int ncS = 2 * P.pS + 1, nv = 2 * (P.pS + P.pD) + 1;
        cd* wsm = sm + (threadIdx.x >> 5) * ((P.down ? ncS : 4 * ncS) + nv);
        if (P.down) fam_dn(gw / P.fch, gw % P.fch, P, col0, col1, wsm);
        else fam_up(gw / P.fch, gw % P.fch, P, col0, col1, wsm);
    } else {
        b -= fb;
        translate_dst(b / P.nch, b % P.nch, P, col0, col1, sm);
    }
}
__global__ void __launch_bounds__(128) k_translate(const XPass P, int nrhs) {
    extern __shared__ cd xsm[];
    // blockIdx.z: a group of columns (the columns of a block right-hand side split over CTAs)
    const int cpb = (nrhs + gridDim.z - 1) / gridDim.z;
    const int col0 = blockIdx.z * cpb, col1 = min(nrhs, col0 + cpb);
    translate_item(blockIdx.x, P, col0, col1, xsm);
}

// Reaction M2L moment tables of components whose source and field layers are the
// same (k_S = k_T, so u = v on every node): I_{mn} = h_{n-m} with
// h_d = sum_q (Fp_q u_q^d + Fm_q u_q^-d), d = -2p..2p -- 4p+1 moments per key
// instead of (2p+1)^2.  One CTA per key; the table is then written out dense.  The
// weights are folded into the power rows, each run of 32 starting from F u^d0 formed
// with a separate exponent (xpow_times): far along the rays u^d alone leaves the double
// range (|u| ~ 2 lambda / k) where F u^d does not, and F = 0 there must not meet u^d = inf.
#define TAB_SAME_CH 8
__global__ void __launch_bounds__(256) k_react_tables_same(MediumDev med, QuadRule q,
                                                           const ReactKey* __restrict__ keys,
                                                           const int* __restrict__ key_list,
                                                           const int* __restrict__ comp, cd* __restrict__ out) {
    extern __shared__ cd sh[];
    const ReactKey K = keys[key_list[blockIdx.x]];
    const int c = K.comp;
    const int ls = comp[4 * c], a = comp[4 * c + 1], lt = comp[4 * c + 2], b = comp[4 * c + 3];
    const int p = K.pS, nco = 2 * p + 1, nd = 4 * p + 1;
    const double ka = med.k[ls];
    // nodes in batches of NB = 256 (all threads evaluate the spectral density, one
    // node each), then in chunks of CH for the power rows and the moment sums
    const int CH = TAB_SAME_CH, NB = 256;
    cd* Pp = sh;                 // [CH][nd]  Fp u^(d - 2p)
    cd* Pm = Pp + CH * nd;       // [CH][nd]  Fm u^(2p - d)
    cd* Fp = Pm + CH * nd;       // [NB]
    cd* Fm = Fp + NB;            // [NB]
    cd* uu = Fm + NB;            // [NB]
    cd* hs = uu + NB;            // [nd] moments
    double h;
    const int P = table_panels(q, K.X, K.D, &h) * q.tab_panel_mult + 2 * p;
    const int ntot = P * 8 + 2 * q.tab_nes;
    const int nseg = (nd + 31) / 32;   // runs of 32 consecutive powers per node and side
    cd acc[2] = {mk(0, 0), mk(0, 0)};   // d = threadIdx.x and threadIdx.x + 256
    for (int jb = 0; jb < ntot; jb += NB) {
        const int cntB = min(NB, ntot - jb);
        __syncthreads();
        if (threadIdx.x < cntB) {
            QuadNode nd2 = table_contour_node(q, jb + threadIdx.x, P, h, K.X, K.D);
            cd S = sigma_comp(med, nd2.lam, ls, a, lt, b);
            cd kya = ky_of(ka, nd2.lam);
            cd SE = S * (eikh(kya, K.hS) * eikh(kya, K.hT));
            Fp[threadIdx.x] = SE * nd2.fp;
            Fm[threadIdx.x] = SE * nd2.fm;
            uu[threadIdx.x] = w_of(kya, nd2.lam, ka);
        }
        for (int j0 = 0; j0 < cntB; j0 += CH) {
            const int cnt = min(CH, cntB - j0);
            __syncthreads();
            // one thread per run of 32: its first value F u^e0 on scaled values, then 31 products
            for (int e = threadIdx.x; e < cnt * 2 * nseg; e += blockDim.x) {
                const int r = e / (2 * nseg), w = e - r * 2 * nseg, side = w / nseg, d0 = (w - side * nseg) * 32;
                const cd u = uu[j0 + r];
                const int e0 = side == 0 ? d0 - 2 * p : 2 * p - d0;
                cd cur = xval(xpow_times(side == 0 ? Fp[j0 + r] : Fm[j0 + r], u, e0));
                const cd step = side == 0 ? u : cinv(u);
                cd* row = (side == 0 ? Pp : Pm) + r * nd;
                const int d1 = min(nd, d0 + 32);
                for (int d = d0; d < d1; ++d) { row[d] = cur; cur = cur * step; }
            }
            __syncthreads();
            for (int s2 = 0; s2 < 2; ++s2) {
                const int di = threadIdx.x + 256 * s2;
                if (di >= nd) break;
                cd ac = acc[s2];
                for (int r = 0; r < cnt; ++r) {
                    ac += Pp[r * nd + di];   // Fp u^d
                    ac += Pm[r * nd + di];   // Fm u^-d
                }
                acc[s2] = ac;
            }
        }
    }
    for (int s2 = 0; s2 < 2; ++s2) {
        const int di = threadIdx.x + 256 * s2;
        if (di < nd) hs[di] = acc[s2];
    }
    __syncthreads();
    // I_{mn} = h_{n-m}, column-major (m, n) at (n + p) nco + (m + p)
    for (int e = threadIdx.x; e < nco * nco; e += blockDim.x) {
        const int ni = e / nco, mi = e - ni * nco;
        out[K.off + e] = hs[(ni - mi) + 2 * p];
    }
}

// Reaction M2L moment tables (eq. generalintegral) of the cross-layer components:
//     I_mn = sum_q [ F+_q v_q^-m u_q^n + F-_q v_q^m u_q^-n ]
// over the table rule's nodes q (u = w(k_a), v = w(k_b), F+- the weights with the spectral
// density and the height factors).  One CTA per run of consecutive entries of one table
// (column-major, (m, n) at (n + pS) ncT + (m + pT)); each thread keeps up to TAB_KPER of them
// in registers.  Per chunk of TAB_CH nodes the CTA stores the powers v^k (k = -pT..pT, one
// table serves both v^-m and v^m) and, for its columns, F+ u^n and F- u^-n (the weights folded
// in), so each entry costs two complex multiply-adds per node and nothing else: the FP64 pipe,
// which bounds the kernel, does only the sum itself, apart from the powers and node values
// (a few per cent).
#define TAB_KPER 16
#define TAB_CH 8
#define TAB_NB 128
struct TableChunk {
    int key;
    int e0, e1;   // entry range [e0, e1) of the key's table, e1 - e0 <= 256 TAB_KPER
};
// dynamic shared memory of one chunk: TAB_CH x (ncT + 2 ncols) powers + 4 TAB_NB node values
__host__ __device__ inline size_t table_chunk_smem(int ncT, int ncols) {
    return (size_t)(TAB_CH * (ncT + 2 * ncols) + 4 * TAB_NB) * sizeof(cd);
}

__global__ void __launch_bounds__(256) k_react_tables(MediumDev med, QuadRule q, const ReactKey* __restrict__ keys,
                                                      const TableChunk* __restrict__ work,
                                                      const int* __restrict__ comp, cd* __restrict__ out) {
    extern __shared__ cd st[];
    const TableChunk wk = work[blockIdx.x];
    const ReactKey K = keys[wk.key];
    const int c = K.comp;
    const int ls = comp[4 * c], a = comp[4 * c + 1], lt = comp[4 * c + 2], b = comp[4 * c + 3];
    const int pS = K.pS, pT = K.pT;
    const int ncT = 2 * pT + 1;
    const double ka = med.k[ls], kb = med.k[lt];
    const int nlo = wk.e0 / ncT, nhi = (wk.e1 - 1) / ncT;   // column indices (from -pS) of the run
    const int ncols = nhi - nlo + 1;
    cd* Wv = st;                          // [TAB_CH][ncT]    v^(k - pT)
    cd* Up = Wv + TAB_CH * ncT;           // [TAB_CH][ncols]  F+ u^n,  n = nlo + j - pS
    cd* Um = Up + TAB_CH * ncols;         // [TAB_CH][ncols]  F- u^-n
    cd* Fp = Um + TAB_CH * ncols;         // [TAB_NB]
    cd* Fm = Fp + TAB_NB;                 // [TAB_NB]
    cd* uu = Fm + TAB_NB;                 // [TAB_NB] u
    cd* vv = uu + TAB_NB;                 // [TAB_NB] v
    // this thread's entries: e = e0 + threadIdx.x + 256 k; row mi and column j within the run
    const int kper = (wk.e1 - wk.e0 + 255) / 256;
    int rowc[TAB_KPER], colc[TAB_KPER];
#pragma unroll
    for (int k = 0; k < TAB_KPER; ++k) {
        const int e = min(wk.e0 + (int)threadIdx.x + 256 * k, wk.e1 - 1);
        rowc[k] = e % ncT;
        colc[k] = e / ncT - nlo;
    }
    double h;
    const int P = table_panels(q, K.X, K.D, &h) * q.tab_panel_mult + (pS + pT);
    const int ntot = P * 8 + 2 * q.tab_nes;
    cd acc[TAB_KPER];
#pragma unroll
    for (int k = 0; k < TAB_KPER; ++k) acc[k] = mk(0, 0);
    const int wruns = (ncT + 31) / 32, uruns = (ncols + 31) / 32;
    for (int jb = 0; jb < ntot; jb += TAB_NB) {
        const int cntB = min(TAB_NB, ntot - jb);
        __syncthreads();
        if (threadIdx.x < cntB) {
            QuadNode nd = table_contour_node(q, jb + threadIdx.x, P, h, K.X, K.D);
            cd S = sigma_comp(med, nd.lam, ls, a, lt, b);
            cd kya = ky_of(ka, nd.lam), kyb = ky_of(kb, nd.lam);
            cd SE = S * (eikh(kya, K.hS) * eikh(kyb, K.hT));
            const cd fp = SE * nd.fp, fm = SE * nd.fm;
            Fp[threadIdx.x] = fp;
            Fm[threadIdx.x] = fm;
            // a node whose weights vanish (far along a ray) adds nothing: powers of 1 keep
            // its finite-valued rows from meeting an infinite power
            const bool zero = fp.x == 0.0 && fp.y == 0.0 && fm.x == 0.0 && fm.y == 0.0;
            uu[threadIdx.x] = zero ? mk(1.0, 0.0) : w_of(kya, nd.lam, ka);
            vv[threadIdx.x] = zero ? mk(1.0, 0.0) : w_of(kyb, nd.lam, kb);
        }
        for (int j0 = 0; j0 < cntB; j0 += TAB_CH) {
            const int cnt = min(TAB_CH, cntB - j0);
            __syncthreads();
            // powers in runs of 32, one thread per run: the run's first power by binary
            // exponentiation, then 31 products (the weights folded into the u runs)
            const int nrun = cnt * (wruns + 2 * uruns);
            for (int t = threadIdx.x; t < nrun; t += blockDim.x) {
                const int r = t / (wruns + 2 * uruns), w = t - r * (wruns + 2 * uruns);
                cd base, fac;
                int e0, len;
                cd* dst;
                bool inv = false;
                if (w < wruns) {                       // v^(k - pT), k = 32 w ..
                    base = vv[j0 + r]; fac = mk(1.0, 0.0);
                    e0 = 32 * w - pT; len = min(32, ncT - 32 * w); dst = Wv + r * ncT + 32 * w;
                } else {
                    const int w2 = w - wruns, sgn = w2 & 1, run = w2 >> 1;
                    base = uu[j0 + r];
                    const int n0 = nlo + 32 * run - pS;
                    len = min(32, ncols - 32 * run);
                    if (sgn == 0) { fac = Fp[j0 + r]; e0 = n0; dst = Up + r * ncols + 32 * run; }
                    else { fac = Fm[j0 + r]; e0 = -n0; dst = Um + r * ncols + 32 * run; inv = true; }
                }
                const cd step = inv ? cinv(base) : base;
                cd cur = xval(xpow_times(fac, base, e0));   // on scaled values: no overflow on the way
                for (int s2 = 0; s2 < len; ++s2) { dst[s2] = cur; cur = cur * step; }
            }
            __syncthreads();
            for (int r = 0; r < cnt; ++r) {
                const cd* W = Wv + r * ncT;
                const cd* P1 = Up + r * ncols;
                const cd* P2 = Um + r * ncols;
#pragma unroll
                for (int k = 0; k < TAB_KPER; ++k) {
                    if (k < kper) {
                        cfma(acc[k], W[2 * pT - rowc[k]], P1[colc[k]]);   // F+ v^-m u^n
                        cfma(acc[k], W[rowc[k]], P2[colc[k]]);            // F- v^m u^-n
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < TAB_KPER; ++k) {
        const int e = wk.e0 + (int)threadIdx.x + 256 * k;
        if (k < kper && e < wk.e1) out[K.off + e] = acc[k];
    }
}

}  // namespace lfmm
