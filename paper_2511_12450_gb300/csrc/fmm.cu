// fmm.cu -- set-up and application of the far field (Sec. 4.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <stdexcept>
#include <tuple>
#include <vector>

#include "fmm_kernels.cuh"
#include "geometry.h"

namespace lfmm {

// Toeplitz vectors of the Graf shifts: J_k(k rho) e^{sgn i k theta}, k in [-hw, hw]
static void graf_j_vector(double k, double dx, double dy, int hw, int sgn, cd* out) {
    double rho = std::hypot(dx, dy);
    double th = std::atan2(dy, dx);
    std::vector<double> J(hw + 1);
    bessel_j_seq(k * rho, hw, J.data());
    for (int kk = -hw; kk <= hw; ++kk) {
        int a = kk < 0 ? -kk : kk;
        double jv = J[a];
        if (kk < 0 && (a & 1)) jv = -jv;
        double ph = sgn * kk * th;
        out[kk + hw] = mk(jv * std::cos(ph), jv * std::sin(ph));
    }
}

// free-space M2L Toeplitz vectors (i/4) H_k(k R) e^{i k Theta}, k in [-2p, 2p]
__global__ void k_m2lf_tables(MediumDev m, const int* __restrict__ tl, const int* __restrict__ tlev,
                              const int* __restrict__ tdx, const int* __restrict__ tdy, const int* __restrict__ tp,
                              const double* __restrict__ tw, const int64_t* __restrict__ toff, int ntab,
                              cd* __restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntab) return;
    const int p2 = 2 * tp[t];
    const double w = tw[t];
    const double dx = tdx[t] * w, dy = tdy[t] * w;
    const double R = hypot(dx, dy), Th = atan2(dy, dx);
    const double z = m.k[tl[t]] * R;
    cd* o = out + toff[t];
    cd hm1 = mk(j0(z), y0(z));
    cd h = mk(j1(z), y1(z));
    for (int kk = 0; kk <= p2; ++kk) {
        cd hk;
        if (kk == 0) hk = hm1;
        else if (kk == 1) hk = h;
        else {
            cd hn = mk((2.0 * (kk - 1) / z) * h.x - hm1.x, (2.0 * (kk - 1) / z) * h.y - hm1.y);
            hm1 = h;
            h = hn;
            hk = hn;
        }
        double s, c;
        sincos(kk * Th, &s, &c);
        cd v = mk(0.0, 0.25) * hk * mk(c, s);       // (i/4) H_k e^{i k Theta}
        o[kk + p2] = v;
        // H_{-k} e^{-i k Theta} = (-1)^k H_k e^{-i k Theta}
        cd vn = mk(0.0, 0.25) * hk * mk(c, -s);
        if (kk & 1) vn = -vn;
        o[-kk + p2] = vn;
    }
}

void fmm_build(lfmm_geometry_s* g) {
    TreeHost& t = g->tree;
    const int D = t.D, l0 = t.l0;
    const int nlev = D + 1;
    const int nl = g->m.nl;
    g->d_p_level = dupload(g, t.p_level);
    // coefficient layout
    std::vector<int64_t> off(t.nbox, -1);
    int64_t nc = 0;
    for (int b = 0; b < t.nbox; ++b) {
        int l = t.box_level[b];
        if (l >= l0) { off[b] = nc; nc += 2 * t.p_level[l] + 1; }
    }
    g->ncoef = nc;
    g->d_coef_off = dupload(g, off);
    if (l0 > D) return;   // no far field: everything is in the near field

    // Reaction centres of cells that straddle their layer's interfaces: the
    // centre of the part of the cell on the layer's side (one slot per
    // (box, side); side 0 = the layer's bottom interface, 1 = its top one).
    // Straddling boxes keep their reaction expansions about these centres:
    // multipoles by a direct P2M from the box's points, locals passed down the
    // tree centre to centre and evaluated at the leaves from there -- never
    // translated to the cell centre, which lies on the far side of the interface.
    {
        std::vector<int> slot_of(2 * t.nbox, -1), slot_box, slot_side;
        std::vector<int64_t> slot_coef;
        std::vector<double> slot_cy;
        int64_t sc = 0;
        const int L = g->m.nl - 1;
        for (int b = t.level_start[l0]; b < t.nbox; ++b) {
            int l = t.box_level[b], lay = t.box_layer[b], p = t.p_level[l];
            double w = t.width(l);
            double lo = t.y0 + t.box_iy[b] * w, hi = t.y0 + (t.box_iy[b] + 1) * w;
            for (int side = 0; side < 2; ++side) {
                if (side == 0 && lay >= L) continue;
                if (side == 1 && lay <= 0) continue;
                double yI = (side == 0) ? g->m.yint[lay] : g->m.yint[lay - 1];
                if (!(lo < yI && yI < hi)) continue;
                double ynew = (side == 0) ? 0.5 * (std::max(lo, yI) + hi) : 0.5 * (lo + std::min(hi, yI));
                slot_of[2 * b + side] = (int)slot_box.size();
                slot_box.push_back(b);
                slot_side.push_back(side);
                slot_cy.push_back(ynew);
                slot_coef.push_back(sc);
                sc += 2 * p + 1;
            }
        }
        g->n_slots = (int)slot_box.size();
        g->nslotcoef = sc;
        g->d_slot_of = dupload(g, slot_of);
        g->d_slot_coef = dupload(g, slot_coef);
        // P2M entries: leaves about cell centres, straddling boxes about reaction centres
        std::vector<ExpEntry> leaf_e, slot_e, slot_leaf_e;
        for (int b = t.level_start[D]; b < t.level_start[D + 1]; ++b)
            leaf_e.push_back(ExpEntry{t.box_begin[b], t.box_end[b], t.box_layer[b], t.p_level[D], t.cx(b), t.cy(b), off[b]});
        for (int q = 0; q < g->n_slots; ++q) {
            int b = slot_box[q];
            ExpEntry e{t.box_begin[b], t.box_end[b], t.box_layer[b], t.p_level[t.box_level[b]], t.cx(b), slot_cy[q],
                       slot_coef[q]};
            if (t.box_level[b] == D) { slot_e.push_back(e); slot_leaf_e.push_back(e); }
        }
        // upward translations into the reaction centres of straddling non-leaf boxes,
        // one list per (parent level, side)
        {
            std::vector<M2MSlot> par;
            std::vector<M2MChild> chl;
            std::vector<cd> vecs;
            g->m2m_slot_start.assign((D + 2) * 2, 0);
            for (int l = l0; l < D; ++l) {
                for (int side = 0; side < 2; ++side) {
                    g->m2m_slot_start[l * 2 + side] = (int)par.size();
                    for (int b = t.level_start[l]; b < t.level_start[l + 1]; ++b) {
                        int sp = slot_of[2 * b + side];
                        if (sp < 0) continue;
                        M2MSlot P;
                        P.pP = t.p_level[l];
                        P.dst_off = slot_coef[sp];
                        P.child_begin = (int)chl.size();
                        for (int c = t.child_begin[b]; c < t.child_end[b]; ++c) {
                            int sc2 = slot_of[2 * c + side];
                            M2MChild C;
                            C.pC = t.p_level[l + 1];
                            C.src_in_slots = (sc2 >= 0) ? 1 : 0;
                            C.src_off = (sc2 >= 0) ? slot_coef[sc2] : off[c];
                            double dx = t.cx(c) - t.cx(b);
                            double dy = (sc2 >= 0 ? slot_cy[sc2] : t.cy(c)) - slot_cy[sp];
                            int hw = P.pP + C.pC;
                            C.vec_off = (int64_t)vecs.size();
                            std::vector<cd> v(2 * hw + 1);
                            graf_j_vector(g->m.k[t.box_layer[b]], dx, dy, hw, -1, v.data());
                            vecs.insert(vecs.end(), v.begin(), v.end());
                            chl.push_back(C);
                        }
                        P.child_end = (int)chl.size();
                        par.push_back(P);
                    }
                }
            }
            g->m2m_slot_start[D * 2] = (int)par.size();
            g->m2m_slot_start[D * 2 + 1] = (int)par.size();
            g->d_m2m_slots = dupload(g, par);
            g->d_m2m_children = dupload(g, chl);
            g->d_m2m_vecs = dupload(g, vecs);
        }
        g->n_leaf_entries = (int)leaf_e.size();
        g->n_slot_entries = (int)slot_e.size();
        g->n_slot_leaf_entries = (int)slot_leaf_e.size();
        g->d_leaf_entries = dupload(g, leaf_e);
        g->d_slot_entries = dupload(g, slot_e);
        g->d_slot_leaf_entries = dupload(g, slot_leaf_e);
        // L2L tasks from the reaction centre of a straddling parent to its children
        // (to the child's reaction centre if it straddles the same interface, else
        // to its cell centre), one list per (level, side)
        std::vector<L2LTask> tasks;
        std::vector<cd> vecs;
        g->task_start.assign((D + 2) * 2, 0);
        for (int l = l0 + 1; l <= D; ++l) {
            for (int side = 0; side < 2; ++side) {
                g->task_start[l * 2 + side] = (int)tasks.size();
                for (int b = t.level_start[l]; b < t.level_start[l + 1]; ++b) {
                    int P = t.box_parent[b];
                    int sp = slot_of[2 * P + side];
                    if (sp < 0) continue;
                    int sb = slot_of[2 * b + side];
                    int pP = t.p_level[l - 1], pC = t.p_level[l];
                    double ux = t.cx(b) - t.cx(P);
                    double uy = (sb >= 0 ? slot_cy[sb] : t.cy(b)) - slot_cy[sp];
                    int hw = pP + pC;
                    L2LTask tk;
                    tk.pS = pP; tk.pD = pC;
                    tk.src_off = slot_coef[sp];
                    tk.src_in_slots = 1;
                    tk.dst_off = (sb >= 0) ? slot_coef[sb] : off[b];
                    tk.dst_in_slots = (sb >= 0) ? 1 : 0;
                    tk.vec_off = (int64_t)vecs.size();
                    std::vector<cd> v(2 * hw + 1);
                    graf_j_vector(g->m.k[t.box_layer[b]], ux, uy, hw, +1, v.data());
                    vecs.insert(vecs.end(), v.begin(), v.end());
                    tasks.push_back(tk);
                }
            }
        }
        g->task_start[(D + 1) * 2] = (int)tasks.size();
        g->task_start[(D + 1) * 2 + 1] = (int)tasks.size();
        g->n_l2l_tasks = (int)tasks.size();
        g->d_l2l_tasks = dupload(g, tasks);
        g->d_l2l_vecs = dupload(g, vecs);
    }

    // M2M and L2L tables per (layer, child level, quadrant)
    {
        std::vector<int64_t> toff(nl * nlev * 4, -1);
        std::vector<cd> m2m, l2l;
        for (int lay = 0; lay < nl; ++lay)
            for (int l = l0 + 1; l <= D; ++l) {
                int hw = t.p_level[l - 1] + t.p_level[l];
                double w = t.width(l);
                for (int quad = 0; quad < 4; ++quad) {
                    double dx = (quad & 1) ? 0.5 * w : -0.5 * w;
                    double dy = (quad & 2) ? 0.5 * w : -0.5 * w;
                    toff[(lay * nlev + l) * 4 + quad] = (int64_t)m2m.size();
                    std::vector<cd> v(2 * hw + 1);
                    graf_j_vector(g->m.k[lay], dx, dy, hw, -1, v.data());   // J_k e^{-i k theta_d}
                    m2m.insert(m2m.end(), v.begin(), v.end());
                    graf_j_vector(g->m.k[lay], dx, dy, hw, +1, v.data());   // J_k e^{+i k theta_u}
                    l2l.insert(l2l.end(), v.begin(), v.end());
                }
            }
        g->d_m2m = dupload(g, m2m);
        g->d_l2l = dupload(g, l2l);
        g->d_m2m_off = dupload(g, toff);
        g->d_l2l_off = g->d_m2m_off;
    }
    // free-space M2L tables per (layer, level, offset) and the V lists with table ids
    {
        std::vector<int> tl, tlev, tdx, tdy, tp;
        std::vector<double> tw;
        std::vector<int64_t> toff;
        std::map<std::tuple<int, int, int, int>, int> id;
        int64_t tot = 0;
        std::vector<int> vf_ptr(t.nbox + 1, 0), vf_src, vf_tab;
        for (int T = 0; T < t.nbox; ++T) {
            for (int e = t.vfree_ptr[T]; e < t.vfree_ptr[T + 1]; ++e) {
                int S = t.vfree_idx[e];
                int l = t.box_level[T], lay = t.box_layer[T];
                int dx = t.box_ix[T] - t.box_ix[S], dy = t.box_iy[T] - t.box_iy[S];
                auto key = std::make_tuple(lay, l, dx, dy);
                auto it = id.find(key);
                int tabid;
                if (it == id.end()) {
                    tabid = (int)tl.size();
                    id[key] = tabid;
                    tl.push_back(lay); tlev.push_back(l); tdx.push_back(dx); tdy.push_back(dy);
                    tp.push_back(t.p_level[l]); tw.push_back(t.width(l));
                    toff.push_back(tot);
                    tot += 4 * t.p_level[l] + 1;
                } else {
                    tabid = it->second;
                }
                vf_src.push_back(S);
                vf_tab.push_back(tabid);
            }
            vf_ptr[T + 1] = (int)vf_src.size();
        }
        g->d_m2lf = dalloc<cd>(g, (size_t)std::max<int64_t>(tot, 1));
        g->d_m2lf_off = dupload(g, toff);
        g->d_vf_ptr = dupload(g, vf_ptr);
        g->d_vf_src = dupload(g, vf_src);
        g->d_vf_tab = dupload(g, vf_tab);
        int ntab = (int)tl.size();
        if (ntab > 0) {
            int* d_tl = dupload(g, tl); int* d_tlev = dupload(g, tlev);
            int* d_tdx = dupload(g, tdx); int* d_tdy = dupload(g, tdy); int* d_tp = dupload(g, tp);
            double* d_tw = dupload(g, tw);
            k_m2lf_tables<<<(ntab + 127) / 128, 128>>>(g->m, d_tl, d_tlev, d_tdx, d_tdy, d_tp, d_tw,
                                                       g->d_m2lf_off, ntab, g->d_m2lf);
            cuda_check(cudaGetLastError(), "k_m2lf_tables");
        }
    }
    // reaction M2L keys, tables and lists
    {
        std::map<std::tuple<int, int, int, int, int>, int> id;
        std::vector<ReactKey> keys;
        std::vector<int> vr_ptr(t.nbox + 1, 0), vr_src, vr_key, vr_comp;
        int64_t tot = 0;
        for (int T = 0; T < t.nbox; ++T) {
            for (int e = t.vreact_ptr[T]; e < t.vreact_ptr[T + 1]; ++e) {
                int S = t.vreact_idx[e], c = t.vreact_comp[e];
                int l = t.box_level[T];
                auto key = std::make_tuple(c, l, t.box_ix[S] - t.box_ix[T], t.box_iy[S], t.box_iy[T]);
                auto it = id.find(key);
                int kid;
                if (it == id.end()) {
                    kid = (int)keys.size();
                    id[key] = kid;
                    const Component& C = t.comps[c];
                    ReactKey rk;
                    rk.comp = c; rk.level = l; rk.pS = t.p_level[l]; rk.pT = t.p_level[l];
                    double w = t.width(l);
                    rk.X = (t.box_ix[S] - t.box_ix[T]) * w;
                    double loS = t.y0 + t.box_iy[S] * w, hiS = t.y0 + (t.box_iy[S] + 1) * w;
                    double loT = t.y0 + t.box_iy[T] * w, hiT = t.y0 + (t.box_iy[T] + 1) * w;
                    rk.hS = src_height_box(g->m, C.ls, C.a, loS, hiS);
                    rk.hT = tgt_height_box(g->m, C.lt, C.b, loT, hiT);
                    rk.D = rk.hS + rk.hT + C.Hc;
                    rk.off = tot;
                    tot += (int64_t)(2 * rk.pT + 1) * (2 * rk.pS + 1);
                    keys.push_back(rk);
                } else {
                    kid = it->second;
                }
                vr_src.push_back(S); vr_key.push_back(kid); vr_comp.push_back(c);
            }
            vr_ptr[T + 1] = (int)vr_src.size();
        }
        g->n_rkeys = (int)keys.size();
        g->d_vr_ptr = dupload(g, vr_ptr);
        g->d_vr_src = dupload(g, vr_src);
        g->d_vr_key = dupload(g, vr_key);
        g->d_vr_comp = dupload(g, vr_comp);
        g->d_rkeys = dupload(g, keys);
        g->d_m2lr = dalloc<cd>(g, (size_t)std::max<int64_t>(tot, 1));
        if (!keys.empty()) {
            std::vector<TableWork> work;
            for (int kk = 0; kk < (int)keys.size(); ++kk) {
                int p = keys[kk].pS;
                for (int m0 = -p; m0 <= p; m0 += 32)
                    for (int n0 = -p; n0 <= p; n0 += 32) work.push_back(TableWork{kk, m0, n0});
            }
            TableWork* d_work = dupload(g, work);
            size_t smem = (size_t)(16 * 32 * 4 + 16 * 4) * sizeof(cd);
            k_react_tables<<<(int)work.size(), 256, smem>>>(g->m, g->quad, g->d_rkeys, d_work, g->d_comp,
                                                            g->d_m2lr);
            cuda_check(cudaGetLastError(), "k_react_tables");
        }
    }
    cuda_check(cudaDeviceSynchronize(), "fmm_build");
}

static void set_smem_limits() {
    static bool done = false;
    if (done) return;
    const int lim = 200 * 1024;
    cuda_check(cudaFuncSetAttribute(k_p2m, cudaFuncAttributeMaxDynamicSharedMemorySize, lim), "smem p2m");
    cuda_check(cudaFuncSetAttribute(k_l2p, cudaFuncAttributeMaxDynamicSharedMemorySize, lim), "smem l2p");
    cuda_check(cudaFuncSetAttribute(k_m2l, cudaFuncAttributeMaxDynamicSharedMemorySize, lim), "smem m2l");
    done = true;
}

static void ensure_coef(lfmm_geometry_s* g, int nrhs) {
    if (g->coef_cols >= nrhs) return;
    if (g->d_M) { cudaFree(g->d_M); cudaFree(g->d_L); }
    if (g->d_Mp) { cudaFree(g->d_Mp); cudaFree(g->d_Lp); }
    g->d_M = g->d_L = g->d_Mp = g->d_Lp = nullptr;
    cuda_check(cudaMalloc(&g->d_M, sizeof(cd) * std::max<int64_t>(g->ncoef, 1) * nrhs), "cudaMalloc M");
    cuda_check(cudaMalloc(&g->d_L, sizeof(cd) * std::max<int64_t>(g->ncoef, 1) * nrhs), "cudaMalloc L");
    cuda_check(cudaMalloc(&g->d_Mp, sizeof(cd) * std::max<int64_t>(g->nslotcoef, 1) * nrhs), "cudaMalloc Mp");
    cuda_check(cudaMalloc(&g->d_Lp, sizeof(cd) * std::max<int64_t>(g->nslotcoef, 1) * nrhs), "cudaMalloc Lp");
    g->coef_cols = nrhs;
}

void fmm_free(lfmm_geometry_s* g) {
    if (g->d_M) { cudaFree(g->d_M); cudaFree(g->d_L); }
    if (g->d_Mp) { cudaFree(g->d_Mp); cudaFree(g->d_Lp); }
    g->d_M = g->d_L = g->d_Mp = g->d_Lp = nullptr;
    g->coef_cols = 0;
}

void fmm_apply(lfmm_geometry_s* g, const cd* x_sorted, cd* y_sorted, int nrhs, cudaStream_t s) {
    set_smem_limits();
    TreeHost& t = g->tree;
    const int D = t.D, l0 = t.l0, nlev = D + 1;
    if (l0 > D) return;
    ensure_coef(g, nrhs);
    const int pD = t.p_level[D];
    int pmax = 0;
    for (int l = l0; l <= D; ++l) pmax = std::max(pmax, t.p_level[l]);
    {   // P2M: leaves about cell centres, straddling boxes about reaction centres
        prof_begin(g, ST_P2M, s);
        size_t smem = (size_t)(32 * (pD + 1)) * sizeof(double) + (size_t)(32 * (pD + 1) + 32) * sizeof(cd);
        k_p2m<<<g->n_leaf_entries, 128, smem, s>>>(g->d_leaf_entries, g->m, g->d_x, g->d_y, g->d_w, x_sorted, g->n,
                                                   nrhs, g->ncoef, g->d_M);
        cuda_check(cudaGetLastError(), "k_p2m");
        if (g->n_slot_entries > 0) {
            size_t sm2 = (size_t)(32 * (pmax + 1)) * sizeof(double) + (size_t)(32 * (pmax + 1) + 32) * sizeof(cd);
            k_p2m<<<g->n_slot_entries, 128, sm2, s>>>(g->d_slot_entries, g->m, g->d_x, g->d_y, g->d_w, x_sorted,
                                                      g->n, nrhs, g->nslotcoef, g->d_Mp);
            cuda_check(cudaGetLastError(), "k_p2m slots");
        }
        prof_end(g, ST_P2M, s);
    }
    prof_begin(g, ST_M2M, s);
    for (int l = D; l > l0; --l) {   // M2M: children at l -> parents at l-1
        int npar = t.level_start[l] - t.level_start[l - 1];
        int pC = t.p_level[l];
        size_t smem = (size_t)(4 * (2 * pC + 1) + 4 * (2 * t.p_level[l - 1] + 1)) * sizeof(cd);
        k_m2m<<<npar, 128, smem, s>>>(t.level_start[l - 1], g->d_child_begin, g->d_child_end, g->d_box_ix,
                                      g->d_box_iy, g->d_box_layer, g->d_coef_off, t.p_level[l - 1], pC, g->d_m2m,
                                      g->d_m2m_off, l, nlev, nrhs, g->ncoef, g->d_M);
        cuda_check(cudaGetLastError(), "k_m2m");
        for (int side = 0; side < 2; ++side) {   // reaction centres of straddling parents at l-1
            int a0 = g->m2m_slot_start[(l - 1) * 2 + side];
            int a1 = (side == 0) ? g->m2m_slot_start[(l - 1) * 2 + 1] : g->m2m_slot_start[l * 2];
            if (a1 > a0) {
                k_m2m_slots<<<a1 - a0, 128, (size_t)(2 * pmax + 1) * sizeof(cd), s>>>(
                    g->d_m2m_slots + a0, g->d_m2m_children, g->d_m2m_vecs, nrhs, g->ncoef, g->nslotcoef, g->d_M,
                    g->d_Mp);
                cuda_check(cudaGetLastError(), "k_m2m_slots");
            }
        }
    }
    prof_end(g, ST_M2M, s);
    {   // M2L, all levels
        prof_begin(g, ST_M2L, s);
        int first = t.level_start[l0];
        int nbx = t.level_start[D + 1] - first;
        size_t smem = (size_t)(M2L_CH * (2 * pmax + 1) + 3 * 4 * (2 * pmax + 1)) * sizeof(cd);
        k_m2l<<<nbx, 128, smem, s>>>(first, g->d_box_level, g->d_p_level, g->d_coef_off, g->d_vf_ptr, g->d_vf_src,
                                     g->d_vf_tab, g->d_m2lf, g->d_m2lf_off, g->d_vr_ptr, g->d_vr_src, g->d_vr_key,
                                     g->d_vr_comp, g->d_comp, g->d_rkeys, g->d_m2lr, nrhs, g->ncoef, g->d_M,
                                     g->d_L, g->d_slot_of, g->d_slot_coef, g->nslotcoef, g->d_Mp, g->d_Lp);
        cuda_check(cudaGetLastError(), "k_m2l");
        prof_end(g, ST_M2L, s);
    }
    prof_begin(g, ST_L2L, s);
    for (int l = l0 + 1; l <= D; ++l) {   // L2L: parents at l-1 -> children at l
        int npar = t.level_start[l] - t.level_start[l - 1];
        int pP = t.p_level[l - 1];
        size_t smem = (size_t)(2 * pP + 1) * sizeof(cd);
        k_l2l<<<npar, 128, smem, s>>>(t.level_start[l - 1], g->d_child_begin, g->d_child_end, g->d_box_ix, g->d_box_iy, g->d_box_layer,
                                     g->d_coef_off, pP, t.p_level[l], g->d_l2l, g->d_l2l_off, l, nlev, nrhs,
                                     g->ncoef, g->d_L);
        cuda_check(cudaGetLastError(), "k_l2l");
        for (int side = 0; side < 2; ++side) {
            int t0 = g->task_start[l * 2 + side];
            int t1 = (side == 0) ? g->task_start[l * 2 + 1] : g->task_start[(l + 1) * 2];
            if (t1 > t0) {
                k_l2l_tasks<<<t1 - t0, 128, (size_t)(2 * pmax + 1) * sizeof(cd), s>>>(
                    g->d_l2l_tasks + t0, g->d_l2l_vecs, nrhs, g->ncoef, g->nslotcoef, g->d_L, g->d_Lp);
                cuda_check(cudaGetLastError(), "k_l2l_tasks");
            }
        }
    }
    prof_end(g, ST_L2L, s);
    {   // L2P: leaves from cell centres, straddling leaves from their reaction centres
        prof_begin(g, ST_L2P, s);
        int threads = 64;
        size_t smem = (size_t)(2 * (2 * pD + 1)) * sizeof(double) + (size_t)threads * (pD + 1) * sizeof(double);
        k_l2p<<<g->n_leaf_entries, threads, smem, s>>>(g->d_leaf_entries, g->m, g->d_x, g->d_y, g->n, nrhs, g->ncoef,
                                                       g->d_L, y_sorted);
        cuda_check(cudaGetLastError(), "k_l2p");
        if (g->n_slot_leaf_entries > 0) {
            k_l2p<<<g->n_slot_leaf_entries, threads, smem, s>>>(g->d_slot_leaf_entries, g->m, g->d_x, g->d_y, g->n,
                                                                nrhs, g->nslotcoef, g->d_Lp, y_sorted);
            cuda_check(cudaGetLastError(), "k_l2p slots");
        }
        prof_end(g, ST_L2P, s);
    }
}

}  // namespace lfmm
