// fmm.cu -- set-up and application of the far field (Sec. 4.1).
//
// Set-up: the free-space Graf shift vectors (multipole-to-multipole as in eq. metome,
// local-to-local as in eq. letole1, multipole-to-local with (i/4) H_{m-n}), the
// reaction components' moment tables I_nm of eq. generalintegral (one per distinct
// box-pair geometry, on the GPU), and the M2L descriptors and work items.
// Application (fmm_apply): P2M (eqs. MEformula, MEcoefficients), M2M, M2L (free space,
// and eq. metoleimage for every reaction component), L2L, L2P (eq. LEformula).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
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

// Groups of consecutive expansion entries for P2M / L2P: at most
// EXP_GROUP_PTS points and EXP_GROUP_ENTRIES entries, or one larger entry.
static std::vector<ExpGroup> make_groups(const std::vector<ExpEntry>& e, int* max_pts, int* max_ent) {
    std::vector<ExpGroup> gs;
    int i = 0;
    while (i < (int)e.size()) {
        ExpGroup G{i, i + 1, e[i].end - e[i].beg};
        while (G.e1 < (int)e.size() && G.e1 - G.e0 < EXP_GROUP_ENTRIES && e[G.e1].p == e[G.e0].p &&
               G.npts + (e[G.e1].end - e[G.e1].beg) <= EXP_GROUP_PTS) {
            G.npts += e[G.e1].end - e[G.e1].beg;
            ++G.e1;
        }
        *max_pts = std::max(*max_pts, G.npts);
        *max_ent = std::max(*max_ent, G.e1 - G.e0);
        gs.push_back(G);
        i = G.e1;
    }
    return gs;
}

// M2L work items over the entry ranges: (box, chunk of output coefficients,
// entry range).  item_work caps the entry x coefficient units of one item (heavy
// (box, chunk)s are split, their parts reduced by k_m2l_reduce); with wide = 1 an
// unsplit box whose coefficients fill a 128-thread CTA better as one row
// (lane_width) gets a single item.  Replaces the geometry's items.
static void make_m2l_items(lfmm_geometry_s* g, int item_work, int wide) {
    TreeHost& t = g->tree;
    const int D = t.D, l0 = t.l0, nlev = D + 1;
    const std::vector<int>& ent_ptr = g->m2l_ent_ptr_host;
    std::vector<M2LItem> items;
    std::vector<M2LReduce> reds;
    int nparts = 0;
    g->m2l_item_level_start.assign(nlev + 2, 0);
    g->m2l_red_level_start.assign(nlev + 2, 0);
    for (int l = l0; l <= D; ++l) {
        g->m2l_item_level_start[l] = (int)items.size();
        g->m2l_red_level_start[l] = (int)reds.size();
        for (int T = t.level_start[l]; T < t.level_start[l + 1]; ++T) {
            const int nco = 2 * t.p_level[l] + 1;
            const int e0 = ent_ptr[T], e1 = ent_ptr[T + 1], ne = e1 - e0;
            const int per = std::max(1, item_work / nco);   // entries per item
            const int np = std::max(1, (ne + per - 1) / per);
            if (wide && np == 1 && lane_width(nco) == nco) {   // one item holds every output coefficient
                items.push_back(M2LItem{T, 0, e0, e1, -1, nco});
                continue;
            }
            for (int c = 0; c * XT_W < nco; ++c) {
                if (np == 1) {
                    items.push_back(M2LItem{T, c, e0, e1, -1, XT_W});
                } else {
                    reds.push_back(M2LReduce{T, c, nparts, np});
                    for (int q = 0; q < np; ++q)
                        items.push_back(M2LItem{T, c, e0 + q * per, std::min(e1, e0 + (q + 1) * per), nparts + q, XT_W});
                    nparts += np;
                }
            }
        }
    }
    for (int l = D + 1; l <= nlev + 1; ++l) {
        g->m2l_item_level_start[l] = (int)items.size();
        g->m2l_red_level_start[l] = (int)reds.size();
    }
    for (int l = 0; l < l0; ++l) { g->m2l_item_level_start[l] = 0; g->m2l_red_level_start[l] = 0; }
    g->n_m2l_items = (int)items.size();
    g->n_m2l_parts = nparts;
    for (void* q : {(void*)g->d_m2l_items, (void*)g->d_m2l_reds}) {   // a schedule being replaced
        auto it = std::find(g->allocs.begin(), g->allocs.end(), q);
        if (q && it != g->allocs.end()) { g->allocs.erase(it); dev_release(q); }
    }
    g->d_m2l_items = dupload(g, items);
    g->d_m2l_reds = dupload(g, reds);
    g->m2l_item_work = item_work;
    g->m2l_wide = wide;
    // the partial-sum buffer is sized for the parts: make the next matvec size it again
    dev_release_now(g->d_m2l_part);
    g->d_m2l_part = nullptr;
    g->m2l_part_cols = 0;
}

// M2L entry descriptors and work items.  Every list entry of a target box
// becomes one M2LEnt (source coefficient offset, table, flags: reaction,
// source in the reaction-centre arrays, arrival/departure directions, output
// array) so the kernels read one descriptor instead of a chain of lookups.
// A work item is (target box, chunk of XT_W outputs, range of entries); the
// entries of a heavy (box, chunk) are split over several items -- at most
// M2L_ITEM_WORK entry x coefficient units each -- whose partial sums a second
// kernel adds in a fixed order, so the few large boxes of the coarse levels
// spread over the GPU instead of running as a handful of long CTAs.
#define M2L_ITEM_WORK 2048
static void build_m2l_work(lfmm_geometry_s* g, const std::vector<int>& vr_ptr, const std::vector<int>& vr_src,
                           const std::vector<int>& vr_key, const std::vector<int>& vr_comp,
                           const std::vector<int>& vr_flip, const std::vector<ReactKey>& keys) {
    TreeHost& t = g->tree;
    std::vector<M2LEnt> ents;
    std::vector<int> ent_ptr(t.nbox + 1, 0);
    for (int T = 0; T < t.nbox; ++T) {
        for (int e = g->vf_ptr_host[T]; e < g->vf_ptr_host[T + 1]; ++e)
            ents.push_back(M2LEnt{g->box_coef_off_host[g->vf_src_host[e]], (int64_t)g->vf_tab_host[e], 0, 0});
        for (int e = vr_ptr[T]; e < vr_ptr[T + 1]; ++e) {
            const int S = vr_src[e];
            const Component& C = t.comps[vr_comp[e]];
            const int a_dir = C.a, b_dir = C.b;
            const int ssl = g->slot_of_host[2 * S + (a_dir == 0 ? 0 : 1)];
            const int side = (b_dir == 0) ? 1 : 0;
            const int dst = (g->slot_of_host[2 * T + side] >= 0) ? 1 + side : 0;
            M2LEnt E;
            E.src = (ssl >= 0) ? g->slot_coef_host[ssl] : g->box_coef_off_host[S];
            E.tab = keys[vr_key[e]].off;
            E.flags = M2L_REACT | (ssl >= 0 ? M2L_SRC_SLOT : 0) | (a_dir ? M2L_A_DOWN : 0) | (b_dir ? M2L_B_DOWN : 0) |
                      (vr_flip[e] ? M2L_FLIP : 0) | (dst << M2L_DST_SHIFT);
            E.pad = 0;
            ents.push_back(E);
        }
        ent_ptr[T + 1] = (int)ents.size();
    }
    g->m2l_ent_ptr_host = ent_ptr;
    g->d_m2l_ents = dupload(g, ents);
    make_m2l_items(g, M2L_ITEM_WORK, 1);
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
    g->box_coef_off_host = off;
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
        g->slot_box_host = slot_box;
        g->slot_coef_host = slot_coef;
        g->nslotcoef = sc;
        g->d_slot_of = dupload(g, slot_of);
        g->slot_of_host = slot_of;
        g->d_slot_coef = dupload(g, slot_coef);
        // P2M entries: leaves about cell centres, straddling boxes about reaction centres
        std::vector<ExpEntry> leaf_e, slot_e, slot_leaf_e;
        for (int b = t.level_start[D]; b < t.level_start[D + 1]; ++b)
            leaf_e.push_back(ExpEntry{t.box_begin[b], t.box_end[b], t.box_layer[b], t.p_level[D], t.cx(b), t.cy(b), off[b],
                                      t.box_begin[b]});
        int64_t brows = g->n;   // basis rows: the points, then each straddling leaf's points again
        for (int q = 0; q < g->n_slots; ++q) {
            int b = slot_box[q];
            ExpEntry e{t.box_begin[b], t.box_end[b], t.box_layer[b], t.p_level[t.box_level[b]], t.cx(b), slot_cy[q],
                       slot_coef[q], brows};
            if (t.box_level[b] == D) {
                slot_e.push_back(e);
                slot_leaf_e.push_back(e);
                brows += t.box_end[b] - t.box_begin[b];
            }
        }
        g->n_leaf_entries = (int)leaf_e.size();
        g->n_slot_entries = (int)slot_e.size();
        g->n_slot_leaf_entries = (int)slot_leaf_e.size();
        {
            int mp = 1, me = 1;
            std::vector<ExpGroup> lg = make_groups(leaf_e, &mp, &me);
            std::vector<ExpGroup> sg = make_groups(slot_e, &mp, &me);
            g->n_leaf_groups = (int)lg.size();
            g->n_slot_groups = (int)sg.size();
            g->d_leaf_groups = dupload(g, lg);
            g->d_slot_groups = dupload(g, sg);
            g->group_max_pts = mp;
            g->group_max_ent = me;
        }
        g->d_leaf_entries = dupload(g, leaf_e);
        g->d_slot_entries = dupload(g, slot_e);
        g->d_slot_leaf_entries = dupload(g, slot_leaf_e);
        // the P2M / L2P basis of every (entry, point), once: J_n(k rho) e^{i n theta} up to the
        // leaf order (one more for the combined field's dipole basis)
        g->basis_ord = t.p_level[D] + (g->combined ? 1 : 0);
        g->d_basis = dalloc<cd>(g, (size_t)brows * (g->basis_ord + 1));
        {
            const size_t smem = (size_t)g->group_max_pts * (g->basis_ord + 1) * sizeof(double);
            raise_smem_limit((const void*)k_basis, smem, "basis smem");
            if (g->n_leaf_groups > 0)
                k_basis<<<g->n_leaf_groups, 128, smem>>>(g->d_leaf_groups, g->d_leaf_entries, g->m, g->d_x, g->d_y,
                                                         g->basis_ord, g->d_basis);
            if (g->n_slot_groups > 0)
                k_basis<<<g->n_slot_groups, 128, smem>>>(g->d_slot_groups, g->d_slot_entries, g->m, g->d_x, g->d_y,
                                                         g->basis_ord, g->d_basis);
            cuda_check(cudaGetLastError(), "k_basis");
        }
        // Upward (M2M) and downward (L2L) passes.  Cells translate as families (a
        // parent and its children, k_translate); each reaction centre of a straddling
        // cell is a destination with its sources and one translation vector per source:
        //   dst_n (= or +=) sum_j sum_m src_j[m] V_j[n - m + pS_j + pD].
        // M2M uses V_k = J_k(k|d|) e^{-i k theta_d} (d = source centre - destination
        // centre); L2L uses J_k(k|u|) e^{+i k theta_u} (u = destination - source)
        // stored reversed, so both passes index n - m.
        std::vector<cd> xvec;
        std::vector<XDst> xd;
        std::vector<XSrc> xs;
        std::vector<int> xd_layer;   // layer of each destination (its sources share it)
        auto put_vec = [&](double k, double dx, double dy, int hw, int sign, bool reverse) -> int64_t {
            std::vector<cd> v(2 * hw + 1);
            graf_j_vector(k, dx, dy, hw, sign, v.data());
            if (reverse) std::reverse(v.begin(), v.end());
            int64_t o = (int64_t)xvec.size();
            xvec.insert(xvec.end(), v.begin(), v.end());
            return o;
        };
        // cell-to-cell base vectors, one per (layer, child level): the quadrant-3 child
        // (+w/2, +w/2); the other quadrants' vectors differ from it by the phases of
        // quarter turns, which the quadrant form applies (fam_up / fam_dn)
        std::vector<int64_t> up_tab(nl * nlev, -1), dn_tab(nl * nlev, -1);
        for (int lay = 0; lay < nl; ++lay)
            for (int l = l0 + 1; l <= D; ++l) {
                int hw = t.p_level[l - 1] + t.p_level[l];
                double w = t.width(l);
                up_tab[lay * nlev + l] = put_vec(g->m.k[lay], 0.5 * w, 0.5 * w, hw, -1, false);
                dn_tab[lay * nlev + l] = put_vec(g->m.k[lay], 0.5 * w, 0.5 * w, hw, +1, true);
            }
        g->qvec_host.assign((size_t)nl * nlev * 2, -1);
        for (int i = 0; i < nl * nlev; ++i) {
            g->qvec_host[2 * i] = up_tab[i];
            g->qvec_host[2 * i + 1] = dn_tab[i];
        }
        auto quad_of = [&](int c) { return (t.box_ix[c] & 1) | ((t.box_iy[c] & 1) << 1); };
        auto slot_y = [&](int b, int sl) { return sl >= 0 ? slot_cy[sl] : t.cy(b); };
        // families: every parent cell at l - 1 with its children at l
        std::vector<QuadX> qx;
        g->q_begin.assign(nlev + 1, 0); g->q_end.assign(nlev + 1, 0);
        for (int l = l0 + 1; l <= D; ++l) {
            g->q_begin[l] = (int)qx.size();
            for (int P = t.level_start[l - 1]; P < t.level_start[l]; ++P) {
                const int lay = t.box_layer[P];
                QuadX f{off[P], {-1, -1, -1, -1}, up_tab[lay * nlev + l], dn_tab[lay * nlev + l], lay, 0};
                for (int c = t.child_begin[P]; c < t.child_end[P]; ++c) {
                    f.ch[quad_of(c)] = off[c];
                    for (int side = 0; side < 2; ++side)
                        if (slot_of[2 * P + side] >= 0 && slot_of[2 * c + side] < 0) f.dn_skip |= 1 << quad_of(c);
                }
                qx.push_back(f);
            }
            g->q_end[l] = (int)qx.size();
        }
        g->up_begin.assign(nlev + 1, 0); g->up_end.assign(nlev + 1, 0);
        g->dn_begin.assign(nlev + 1, 0); g->dn_end.assign(nlev + 1, 0);
        // the remaining destinations: reaction centres of straddling cells, each with its
        // own sources and vectors
        for (int lp = D - 1; lp >= l0; --lp) {   // M2M into parents at level lp
            const int pP = t.p_level[lp], pC = t.p_level[lp + 1], hw = pP + pC;
            g->up_begin[lp] = (int)xd.size();
            for (int side = 0; side < 2; ++side)
                for (int b = t.level_start[lp]; b < t.level_start[lp + 1]; ++b) {
                    const int sp = slot_of[2 * b + side];
                    if (sp < 0) continue;
                    XDst d{slot_coef[sp], pP, 1, (int)xs.size(), 0};
                    for (int c = t.child_begin[b]; c < t.child_end[b]; ++c) {
                        const int sc2 = slot_of[2 * c + side];
                        const int64_t v = put_vec(g->m.k[t.box_layer[b]], t.cx(c) - t.cx(b), slot_y(c, sc2) - slot_cy[sp],
                                                  hw, -1, false);
                        xs.push_back(XSrc{sc2 >= 0 ? slot_coef[sc2] : off[c], v, pC, sc2 >= 0 ? 1 : 0});
                    }
                    d.src_end = (int)xs.size();
                    xd.push_back(d);
                    xd_layer.push_back(t.box_layer[b]);
                }
            g->up_end[lp] = (int)xd.size();
        }
        for (int l = l0 + 1; l <= D; ++l) {   // L2L into children at level l
            const int pP = t.p_level[l - 1], pC = t.p_level[l], hw = pP + pC;
            g->dn_begin[l] = (int)xd.size();
            // cells under a straddling parent that do not straddle that interface: the
            // parent's cell local and its reaction-centre locals
            for (int q = g->q_begin[l]; q < g->q_end[l]; ++q) {
                const int P = t.level_start[l - 1] + (q - g->q_begin[l]);   // one family per parent, in order
                if (!qx[q].dn_skip) continue;
                for (int c = t.child_begin[P]; c < t.child_end[P]; ++c) {
                    if (!((qx[q].dn_skip >> quad_of(c)) & 1)) continue;
                    XDst d{off[c], pC, 0, (int)xs.size(), 0};
                    xs.push_back(XSrc{off[P], put_vec(g->m.k[t.box_layer[c]], t.cx(c) - t.cx(P), t.cy(c) - t.cy(P), hw, +1, true),
                                      pP, 0});
                    for (int side = 0; side < 2; ++side) {
                        const int sp = slot_of[2 * P + side];
                        if (sp < 0 || slot_of[2 * c + side] >= 0) continue;
                        const int64_t v = put_vec(g->m.k[t.box_layer[c]], t.cx(c) - t.cx(P), t.cy(c) - slot_cy[sp], hw, +1, true);
                        xs.push_back(XSrc{slot_coef[sp], v, pP, 1});
                    }
                    d.src_end = (int)xs.size();
                    xd.push_back(d);
                    xd_layer.push_back(t.box_layer[c]);
                }
            }
            for (int side = 0; side < 2; ++side)
                for (int b = t.level_start[l]; b < t.level_start[l + 1]; ++b) {
                    const int sb = slot_of[2 * b + side];
                    if (sb < 0) continue;
                    const int P = t.box_parent[b];
                    const int sp = slot_of[2 * P + side];
                    // a cell that contains the interface lies in a parent that contains it too
                    if (sp < 0) throw CudaError{"internal: straddling cell under a non-straddling parent"};
                    XDst d{slot_coef[sb], pC, 1, (int)xs.size(), 0};
                    const int64_t v = put_vec(g->m.k[t.box_layer[b]], t.cx(b) - t.cx(P), slot_cy[sb] - slot_cy[sp], hw, +1, true);
                    xs.push_back(XSrc{slot_coef[sp], v, pP, 1});
                    d.src_end = (int)xs.size();
                    xd.push_back(d);
                    xd_layer.push_back(t.box_layer[b]);
                }
            g->dn_end[l] = (int)xd.size();
        }
        g->d_qx = dupload(g, qx);
        g->qx_host = qx;
        g->d_xdst = dupload(g, xd);
        g->d_xsrc = dupload(g, xs);
        g->d_xvec = dupload(g, xvec);
        g->xdst_host = xd;
        g->xsrc_host = xs;
        g->xd_layer_host = xd_layer;
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
        g->m2lf_len = tot;
        g->d_m2lf_off = dupload(g, toff);
        g->ftab_lay = tl;
        g->ftab_lev = tlev;
        g->d_vf_ptr = dupload(g, vf_ptr);
        g->d_vf_src = dupload(g, vf_src);
        g->d_vf_tab = dupload(g, vf_tab);
        g->vf_ptr_host = vf_ptr;
        g->vf_src_host = vf_src;
        g->vf_tab_host = vf_tab;
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
        std::vector<int> vr_ptr(t.nbox + 1, 0), vr_src, vr_key, vr_comp, vr_flip;
        int64_t tot = 0;
        for (int T = 0; T < t.nbox; ++T) {
            for (int e = t.vreact_ptr[T]; e < t.vreact_ptr[T + 1]; ++e) {
                int S = t.vreact_idx[e], c = t.vreact_comp[e];
                int l = t.box_level[T];
                // a pair at horizontal offset -X uses the table of +X with both indices
                // reversed: lambda -> -lambda maps e^{i lambda X} to e^{-i lambda X} and
                // w(lambda, k) to 1 / w(lambda, k) (k_y is even in lambda), so
                // I(-X)_{mn} = I(X)_{-m,-n}
                const int dix = t.box_ix[S] - t.box_ix[T];
                const int flip = dix < 0 ? 1 : 0;
                auto key = std::make_tuple(c, l, flip ? -dix : dix, t.box_iy[S], t.box_iy[T]);
                auto it = id.find(key);
                int kid;
                if (it == id.end()) {
                    kid = (int)keys.size();
                    id[key] = kid;
                    const Component& C = t.comps[c];
                    ReactKey rk;
                    rk.comp = c; rk.level = l; rk.pS = t.p_level[l]; rk.pT = t.p_level[l];
                    double w = t.width(l);
                    rk.X = (flip ? -dix : dix) * w;
                    double loS = t.y0 + t.box_iy[S] * w, hiS = t.y0 + (t.box_iy[S] + 1) * w;
                    double loT = t.y0 + t.box_iy[T] * w, hiT = t.y0 + (t.box_iy[T] + 1) * w;
                    rk.hS = src_height_box(g->m, C.ls, C.a, loS, hiS);
                    rk.hT = tgt_height_box(g->m, C.lt, C.b, loT, hiT);
                    rk.D = rk.hS + rk.hT + C.Hc;
                    rk.off = tot;
                    g->rkey_lay_s.push_back(t.box_layer[S]);
                    g->rkey_lay_t.push_back(t.box_layer[T]);
                    tot += (int64_t)(2 * rk.pT + 1) * (2 * rk.pS + 1);
                    keys.push_back(rk);
                } else {
                    kid = it->second;
                }
                vr_src.push_back(S); vr_key.push_back(kid); vr_comp.push_back(c); vr_flip.push_back(flip);
            }
            vr_ptr[T + 1] = (int)vr_src.size();
        }
        g->n_rkeys = (int)keys.size();
        g->d_vr_ptr = dupload(g, vr_ptr);
        g->d_vr_src = dupload(g, vr_src);
        g->d_vr_key = dupload(g, vr_key);
        g->d_vr_comp = dupload(g, vr_comp);
        build_m2l_work(g, vr_ptr, vr_src, vr_key, vr_comp, vr_flip, keys);
        g->d_rkeys = dupload(g, keys);
        g->rkeys_host = keys;
        g->d_m2lr = dalloc<cd>(g, (size_t)std::max<int64_t>(tot, 1));
        g->m2lr_len = tot;
        if (!keys.empty()) {
            // same-layer components: Toeplitz tables from 4p+1 moments; others in runs of entries
            std::vector<TableChunk> work;
            std::vector<int> same;
            int pmax_same = 0;
            size_t smem = 0;
            for (int kk = 0; kk < (int)keys.size(); ++kk) {
                const Component& C = t.comps[keys[kk].comp];
                int p = keys[kk].pS;
                double hq = 0.0;
                const int P0 = table_panels(g->quad, keys[kk].X, keys[kk].D, &hq) * g->quad.tab_panel_mult;
                if (C.ls == C.lt && keys[kk].pS == keys[kk].pT) {
                    same.push_back(kk);
                    pmax_same = std::max(pmax_same, p);
                    // 4p + 1 moments, two terms per node
                    g->table_cmacs[1] += 2.0 * (4 * p + 1) * ((P0 + 2 * p) * 8.0 + 2 * g->quad.tab_nes);
                    continue;
                }
                // (2pT + 1) (2pS + 1) entries, two terms per node
                const int ncT = 2 * keys[kk].pT + 1, ne = ncT * (2 * keys[kk].pS + 1);
                g->table_cmacs[0] += 2.0 * ne * ((P0 + keys[kk].pS + keys[kk].pT) * 8.0 + 2 * g->quad.tab_nes);
                // runs of nearly equal length, at most 256 TAB_KPER entries each
                const int nch = (ne + 256 * TAB_KPER - 1) / (256 * TAB_KPER);
                for (int ci = 0; ci < nch; ++ci) {
                    const int e0 = (int)((int64_t)ne * ci / nch), e1 = (int)((int64_t)ne * (ci + 1) / nch);
                    work.push_back(TableChunk{kk, e0, e1});
                    smem = std::max(smem, table_chunk_smem(ncT, (e1 - 1) / ncT - e0 / ncT + 1));
                }
            }
            if (!work.empty()) {
                TableChunk* d_work = dupload(g, work);
                raise_smem_limit((const void*)k_react_tables, smem, "reaction tables smem");
                k_react_tables<<<(int)work.size(), 256, smem>>>(g->m, g->quad, g->d_rkeys, d_work, g->d_comp,
                                                                g->d_m2lr);
                cuda_check(cudaGetLastError(), "k_react_tables");
            }
            if (!same.empty()) {
                int* d_same = dupload(g, same);
                const int nd = 4 * pmax_same + 1;
                const size_t smem = (size_t)(2 * TAB_SAME_CH * nd + 3 * 256 + nd) * sizeof(cd);   // k_react_tables_same layout
                raise_smem_limit((const void*)k_react_tables_same, smem, "same-layer tables smem");
                k_react_tables_same<<<(int)same.size(), 256, smem>>>(g->m, g->quad, g->d_rkeys, d_same, g->d_comp,
                                                                     g->d_m2lr);
                cuda_check(cudaGetLastError(), "k_react_tables_same");
            }
        }
    }
    cuda_check(cudaStreamSynchronize(cudaStreamPerThread), "fmm_build");
}

void raise_smem_limit(const void* func, size_t bytes, const char* what) {
    if (bytes <= 48 * 1024) return;   // no opt-in needed
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> granted;
    int dev = 0;
    cuda_check(cudaGetDevice(&dev), what);
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = granted[std::make_pair(func, dev)];
    if (bytes <= cur) return;
    cuda_check(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes), what);
    cur = bytes;
}

static void set_smem_limits() {
    const size_t lim = 200 * 1024;
    raise_smem_limit((const void*)k_p2m, lim, "smem p2m");
    raise_smem_limit((const void*)k_l2p, lim, "smem l2p");
    raise_smem_limit((const void*)k_m2l, lim, "smem m2l");
}

static void ensure_coef(lfmm_geometry_s* g, int nrhs) {
    if (g->coef_cols >= nrhs) return;
    dev_release_now(g->d_M); dev_release_now(g->d_L);
    dev_release_now(g->d_Mp); dev_release_now(g->d_Lp);
    g->d_M = g->d_L = g->d_Mp = g->d_Lp = nullptr;
    g->d_M = (cd*)dev_alloc_ready(sizeof(cd) * std::max<int64_t>(g->ncoef, 1) * nrhs, "M");
    g->d_L = (cd*)dev_alloc_ready(sizeof(cd) * std::max<int64_t>(g->ncoef, 1) * nrhs, "L");
    g->d_Mp = (cd*)dev_alloc_ready(sizeof(cd) * std::max<int64_t>(g->nslotcoef, 1) * nrhs, "Mp");
    g->d_Lp = (cd*)dev_alloc_ready(sizeof(cd) * std::max<int64_t>(g->nslotcoef, 1) * nrhs, "Lp");
    g->coef_cols = nrhs;
}

void fmm_free(lfmm_geometry_s* g) {
    dev_release(g->d_m2l_part);
    g->d_m2l_part = nullptr;
    g->m2l_part_cols = 0;
    dev_release(g->d_M); dev_release(g->d_L);
    dev_release(g->d_Mp); dev_release(g->d_Lp);
    g->d_M = g->d_L = g->d_Mp = g->d_Lp = nullptr;
    g->coef_cols = 0;
}

// FP64 M2L over the first n64 work items and the first r64 reductions of split
// items (the levels below the precision form's first FP32 level, or all levels).
static void ensure_m2l_part(lfmm_geometry_s* g, int nrhs) {
    if (g->n_m2l_parts > 0 && g->m2l_part_cols < nrhs) {
        dev_release_now(g->d_m2l_part);
        g->d_m2l_part = nullptr;
        g->d_m2l_part = (cd*)dev_alloc_ready(sizeof(cd) * (size_t)g->n_m2l_parts * 3 * XT_W * nrhs,
                                             "M2L partial sums");
        g->m2l_part_cols = nrhs;
    }
}
// FP64 M2L of the work items [i0, i1) and the reductions [r0, r1) (a range of levels)
static void launch_m2l_range(lfmm_geometry_s* g, int nrhs, int i0, int i1, int r0, int r1, cudaStream_t s) {
    if (i1 > i0) {
        k_m2l<<<i1 - i0, 128, 0, s>>>(g->d_m2l_items + i0, g->d_m2l_ents, g->d_box_level, g->d_p_level,
                                      g->d_coef_off, g->d_slot_of, g->d_slot_coef, g->d_m2lf, g->d_m2lf_off,
                                      g->d_m2lr, nrhs, g->ncoef, g->nslotcoef, g->n_m2l_parts, g->d_M, g->d_Mp,
                                      g->d_L, g->d_Lp, g->d_m2l_part);
        cuda_check(cudaGetLastError(), "k_m2l");
        ++g->n_launches;
    }
    if (r1 > r0) {
        k_m2l_reduce<<<r1 - r0, 64, 0, s>>>(g->d_m2l_reds + r0, g->d_box_level, g->d_p_level, g->d_coef_off,
                                            g->d_slot_of, g->d_slot_coef, nrhs, g->ncoef, g->nslotcoef,
                                            g->n_m2l_parts, g->d_m2l_part, g->d_L, g->d_Lp);
        cuda_check(cudaGetLastError(), "k_m2l_reduce");
        ++g->n_launches;
    }
}
static void launch_m2l64(lfmm_geometry_s* g, int nrhs, int n64, int r64, cudaStream_t s) {
    ensure_m2l_part(g, nrhs);
    launch_m2l_range(g, nrhs, 0, n64, 0, r64, s);
}

// one level's M2M (into parents at level - 1: down = 0) or L2L (into children at level:
// down = 1) pass over a block of nrhs columns
static XPass make_pass(lfmm_geometry_s* g, int level, int down, int accumulate, int nrhs) {
    const TreeHost& t = g->tree;
    XPass P;
    P.dsts = g->d_xdst + (down ? g->dn_begin[level] : g->up_begin[level - 1]);
    P.srcs = g->d_xsrc;
    P.vec = g->d_xvec;
    P.qx = g->d_qx + g->q_begin[level];
    P.nq = g->q_end[level] - g->q_begin[level];
    P.nd = down ? g->dn_end[level] - g->dn_begin[level] : g->up_end[level - 1] - g->up_begin[level - 1];
    P.pS = down ? t.p_level[level - 1] : t.p_level[level];
    P.pD = down ? t.p_level[level] : t.p_level[level - 1];
    const int nco = 2 * P.pD + 1;
    P.w = lane_width(nco);
    P.nch = (nco + P.w - 1) / P.w;
    xpass_fam_split(P.nq, P.pD, &P.fch, &P.fr);
    P.down = down;
    P.accumulate = accumulate;
    P.ncoef = g->ncoef;
    P.nslotcoef = g->nslotcoef;
    P.X = down ? g->d_L : g->d_M;
    P.Xp = down ? g->d_Lp : g->d_Mp;
    (void)nrhs;
    return P;
}
static void launch_pass(lfmm_geometry_s* g, const XPass& P, int nrhs, cudaStream_t s, const char* what) {
    const int items = xpass_fam_ctas(P.nq, P.fch) + P.nd * P.nch;
    if (items == 0) return;
    const size_t smem = xpass_smem(P.down, P.pS, P.pD, P.w);
    raise_smem_limit((const void*)k_translate, smem, "translate smem");
    k_translate<<<dim3(items, 1, col_groups(nrhs)), 128, smem, s>>>(P, nrhs);
    cuda_check(cudaGetLastError(), what);
    ++g->n_launches;
}

void fmm_apply(lfmm_geometry_s* g, const cd* x_sorted, cd* y_sorted, int nrhs, cudaStream_t s, bool mixed,
               cudaEvent_t before_l2p) {
    set_smem_limits();
    TreeHost& t = g->tree;
    const int D = t.D, l0 = t.l0;
    if (l0 > D) return;
    ensure_coef(g, nrhs);
    const int pD = t.p_level[D];
    int pmax = 0;
    for (int l = l0; l <= D; ++l) pmax = std::max(pmax, t.p_level[l]);
    // shared memory of the grouped P2M / L2P kernels (same order p = p_D for every entry)
    const int gp = g->group_max_pts, ge = g->group_max_ent;
    const int rs_p2m = 2 * (g->combined ? pD + 1 : pD) + 1;   // basis row length (k_p2m)
    const size_t smem_p2m = (size_t)gp * rs_p2m * sizeof(cd) + (size_t)gp * sizeof(cd) + (size_t)(gp + 1) * sizeof(int);
    const size_t smem_l2p = (size_t)ge * 2 * (pD + 1) * sizeof(cd);
    raise_smem_limit((const void*)k_p2m, smem_p2m, "p2m smem");
    raise_smem_limit((const void*)k_l2p, smem_l2p, "l2p smem");
    // precision form: the levels >= lm run in FP32 on scaled expansions (lm > D: none)
    const int lm = mixed ? std::max(l0, std::min(mixed_level(g), D + 1)) : D + 1;
    if (lm <= D) mixed_setup(g, nrhs);
    {   // P2M: leaves about cell centres, straddling leaves about reaction centres
        prof_begin(g, ST_P2M, s);
        if (lm <= D) {
            mixed_p2m(g, x_sorted, nrhs, s);
        } else {
            k_p2m<<<g->n_leaf_groups, 128, smem_p2m, s>>>(g->d_leaf_groups, g->d_leaf_entries, g->m, g->d_w, g->d_nx,
                                                          g->d_ny, g->d_basis, g->basis_ord + 1, x_sorted, g->n, nrhs,
                                                          g->ncoef, g->d_M);
            cuda_check(cudaGetLastError(), "k_p2m");
            ++g->n_launches;
            if (g->n_slot_groups > 0) {
                k_p2m<<<g->n_slot_groups, 128, smem_p2m, s>>>(g->d_slot_groups, g->d_slot_entries, g->m, g->d_w,
                                                              g->d_nx, g->d_ny, g->d_basis, g->basis_ord + 1, x_sorted,
                                                              g->n, nrhs, g->nslotcoef, g->d_Mp);
                cuda_check(cudaGetLastError(), "k_p2m slots");
                ++g->n_launches;
            }
        }
        prof_end(g, ST_P2M, s);
    }
    prof_begin(g, ST_M2M, s);
    for (int lp = D - 1; lp >= l0; --lp) {   // M2M: children at lp + 1 -> parents (cells and reaction centres) at lp
        if (lp >= lm) { mixed_m2m(g, lp, nrhs, s); continue; }
        if (lp == lm - 1) mixed_m_to64(g, lm, nrhs, s);   // the FP64 levels start from the FP32 ones' multipoles
        launch_pass(g, make_pass(g, lp + 1, 0, 0, nrhs), nrhs, s, "k_translate (M2M)");
    }
    prof_end(g, ST_M2M, s);
    {   // M2L, all levels (precision form: the levels >= lm in FP32)
        prof_begin(g, ST_M2L, s);
        const int n64 = g->m2l_item_level_start[lm];
        const int r64 = g->m2l_red_level_start[lm];
        if (lm <= D && mixed_coarse_df(g)) {
            // precision form: the coarse (wide-band) levels in double-float, the rest in FP32
            ensure_m2l_part(g, nrhs);
            mixed_m2l_coarse(g, nrhs, n64, s);
            launch_m2l_range(g, nrhs, 0, 0, 0, r64, s);
        } else {
            launch_m2l64(g, nrhs, n64, r64, s);
        }
        if (lm <= D) mixed_m2l(g, nrhs, lm, s);
        prof_end(g, ST_M2L, s);
    }
    prof_begin(g, ST_L2L, s);
    for (int l = l0 + 1; l <= D; ++l) {   // L2L: parents at l - 1 -> children (cells and reaction centres) at l
        if (l > lm) { mixed_l2l(g, l, nrhs, s); continue; }
        // at the first FP32 level the FP64 translation writes (not adds) and is then added
        // into the FP32 locals, which the FP32 M2L has written
        const int acc = (l == lm) ? 0 : 1;
        launch_pass(g, make_pass(g, l, 1, acc, nrhs), nrhs, s, "k_translate (L2L)");
        if (l == lm) mixed_l_add(g, lm, nrhs, s);
    }
    prof_end(g, ST_L2L, s);
    {   // L2P: leaves from cell centres, straddling leaves from their reaction centres
        // (after the near field, which adds into the same y on the side stream)
        if (before_l2p) cuda_check(cudaStreamWaitEvent(s, before_l2p, 0), "wait for the near field");
        prof_begin(g, ST_L2P, s);
        if (lm <= D) {
            mixed_l2p(g, y_sorted, nrhs, s);
        } else {
            k_l2p<<<g->n_leaf_groups, 128, smem_l2p, s>>>(g->d_leaf_groups, g->d_leaf_entries, g->d_basis,
                                                          g->basis_ord + 1, g->n, nrhs, g->ncoef, g->d_L, y_sorted);
            cuda_check(cudaGetLastError(), "k_l2p");
            ++g->n_launches;
            if (g->n_slot_groups > 0) {
                k_l2p<<<g->n_slot_groups, 128, smem_l2p, s>>>(g->d_slot_groups, g->d_slot_leaf_entries, g->d_basis,
                                                              g->basis_ord + 1, g->n, nrhs, g->nslotcoef, g->d_Lp,
                                                              y_sorted);
                cuda_check(cudaGetLastError(), "k_l2p slots");
                ++g->n_launches;
            }
        }
        prof_end(g, ST_L2P, s);
    }
}

// ------------------------------------------------------------------ batched far field
// Several geometries' far fields in shared launches.  Each launch gets a table of jobs
// (one geometry's arguments for the stage) and the prefix of their block counts; a CTA
// finds its job by binary search over the prefix and runs the same body as the
// single-geometry kernel with its block index within the job, so every geometry's
// result is the one its own launches give, bit for bit.
struct P2MJob {
    const ExpGroup* groups;
    const ExpEntry* ent;
    MediumDev m;
    const double *pw, *nx, *ny;
    const cd* basis;
    int bstride;
    const cd* phi;
    int64_t n, stride;
    int nrhs;
    cd* M;
};
struct L2PJob {
    const ExpGroup* groups;
    const ExpEntry* ent;
    const cd* basis;
    int bstride;
    int64_t n, stride;
    int nrhs;
    const cd* L;
    cd* y;
};
struct XJob {
    XPass P;
    int nrhs;
};
struct M2LJob {
    const M2LItem* items;
    const M2LReduce* reds;
    const M2LEnt* ents;
    const int *box_level, *p_level, *slot_of;
    const int64_t *coef_off, *slot_coef, *m2lf_off;
    const cd *m2lf, *m2lr;
    int nrhs, nparts;
    int64_t ncoef, nslotcoef;
    const cd *M, *Mp;
    cd *L, *Lp, *part;
};

__device__ __forceinline__ int job_of(const int* __restrict__ prefix, int njobs, int b) {
    int lo = 0, hi = njobs - 1;   // the last job whose first block is <= b (jobs without blocks are passed over)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__global__ void __launch_bounds__(128) k_p2m_multi(const P2MJob* __restrict__ jobs, const int* __restrict__ prefix,
                                                   int njobs) {
    const int j = job_of(prefix, njobs, blockIdx.x);
    const P2MJob& J = jobs[j];
    p2m_group(blockIdx.x - prefix[j], J.groups, J.ent, J.m, J.pw, J.nx, J.ny, J.basis, J.bstride, J.phi, J.n, J.nrhs,
              J.stride, J.M);
}
__global__ void __launch_bounds__(128) k_l2p_multi(const L2PJob* __restrict__ jobs, const int* __restrict__ prefix,
                                                   int njobs) {
    const int j = job_of(prefix, njobs, blockIdx.x);
    const L2PJob& J = jobs[j];
    l2p_group(blockIdx.x - prefix[j], J.groups, J.ent, J.basis, J.bstride, J.n, J.nrhs, J.stride, J.L, J.y);
}
__global__ void __launch_bounds__(128) k_translate_multi(const XJob* __restrict__ jobs, const int* __restrict__ prefix,
                                                         int njobs) {
    extern __shared__ cd xsm[];
    const int j = job_of(prefix, njobs, blockIdx.x);
    const XPass P = jobs[j].P;
    translate_item(blockIdx.x - prefix[j], P, 0, jobs[j].nrhs, xsm);
}
__global__ void __launch_bounds__(128) k_m2l_multi(const M2LJob* __restrict__ jobs, const int* __restrict__ prefix,
                                                   int njobs) {
    const int j = job_of(prefix, njobs, blockIdx.x);
    const M2LJob& J = jobs[j];
    m2l_item(blockIdx.x - prefix[j], J.items, J.ents, J.box_level, J.p_level, J.coef_off, J.slot_of, J.slot_coef,
             J.m2lf, J.m2lf_off, J.m2lr, J.nrhs, J.ncoef, J.nslotcoef, J.nparts, J.M, J.Mp, J.L, J.Lp, J.part);
}
__global__ void __launch_bounds__(64) k_m2l_reduce_multi(const M2LJob* __restrict__ jobs,
                                                         const int* __restrict__ prefix, int njobs) {
    const int j = job_of(prefix, njobs, blockIdx.x);
    const M2LJob& J = jobs[j];
    m2l_reduce_one(blockIdx.x - prefix[j], J.reds, J.box_level, J.p_level, J.coef_off, J.slot_of, J.slot_coef,
                   J.nrhs, J.ncoef, J.nslotcoef, J.nparts, J.part, J.L, J.Lp);
}

void JobTables::upload(cudaStream_t s) {
    if (host.empty()) return;
    cuda_check(cudaMallocAsync((void**)&dev, host.size(), s), "cudaMallocAsync job tables");
    // from pageable memory: the call returns once the bytes are staged, so the host
    // vector may change afterwards
    cuda_check(cudaMemcpyAsync(dev, host.data(), host.size(), cudaMemcpyHostToDevice, s), "job tables h2d");
}
void JobTables::release(cudaStream_t s) {
    if (dev) cudaFreeAsync(dev, s);
    dev = nullptr;
}

// One fused launch: jobs of type J with their block counts; no launch without blocks.
template <class J, class K>
static void launch_jobs(const std::vector<J>& jobs, const std::vector<int>& blocks, K kernel, int threads, size_t smem,
                        cudaStream_t s, const char* what) {
    std::vector<int> prefix(jobs.size() + 1, 0);
    for (size_t i = 0; i < jobs.size(); ++i) prefix[i + 1] = prefix[i] + blocks[i];
    if (jobs.empty() || prefix.back() == 0) return;
    JobTables t;
    const size_t oj = t.add(jobs.data(), sizeof(J) * jobs.size());
    const size_t op = t.add(prefix.data(), sizeof(int) * prefix.size());
    t.upload(s);
    kernel<<<prefix.back(), threads, smem, s>>>(t.at<J>(oj), t.at<int>(op), (int)jobs.size());
    cudaError_t e = cudaGetLastError();
    t.release(s);
    cuda_check(e, what);
}

void fmm_apply_batch(const std::vector<BatchOp>& ops, cudaStream_t s, cudaEvent_t before_l2p) {
    set_smem_limits();
    std::vector<const BatchOp*> far;
    size_t smem_p2m = 0, smem_l2p = 0;
    int max_up = 0, max_dn = 0;
    for (const BatchOp& op : ops) {
        lfmm_geometry_s* g = op.g;
        const TreeHost& t = g->tree;
        if (t.l0 > t.D) continue;
        far.push_back(&op);
        ensure_coef(g, op.nrhs);
        if (g->n_m2l_parts > 0 && g->m2l_part_cols < op.nrhs) {
            dev_release_now(g->d_m2l_part);
            g->d_m2l_part = nullptr;
            g->d_m2l_part = (cd*)dev_alloc_ready(sizeof(cd) * (size_t)g->n_m2l_parts * 3 * XT_W * op.nrhs,
                                                 "M2L partial sums");
            g->m2l_part_cols = op.nrhs;
        }
        const int pD = t.p_level[t.D], gp = g->group_max_pts, ge = g->group_max_ent;
        const int rs = 2 * (g->combined ? pD + 1 : pD) + 1;
        smem_p2m = std::max(smem_p2m, (size_t)gp * rs * sizeof(cd) + (size_t)gp * sizeof(cd) + (size_t)(gp + 1) * sizeof(int));
        smem_l2p = std::max(smem_l2p, (size_t)ge * 2 * (pD + 1) * sizeof(cd));
        max_up = std::max(max_up, t.D - t.l0);
        max_dn = std::max(max_dn, t.D - t.l0);
    }
    if (far.empty()) {
        if (before_l2p) cuda_check(cudaStreamWaitEvent(s, before_l2p, 0), "wait for the near field");
        return;
    }
    raise_smem_limit((const void*)k_p2m_multi, smem_p2m, "p2m smem");
    raise_smem_limit((const void*)k_l2p_multi, smem_l2p, "l2p smem");
    {   // P2M: leaves about cell centres, straddling leaves about reaction centres
        std::vector<P2MJob> jobs;
        std::vector<int> blocks;
        for (const BatchOp* op : far) {
            lfmm_geometry_s* g = op->g;
            jobs.push_back(P2MJob{g->d_leaf_groups, g->d_leaf_entries, g->m, g->d_w, g->d_nx, g->d_ny, g->d_basis,
                                  g->basis_ord + 1, op->x, g->n, g->ncoef, op->nrhs, g->d_M});
            blocks.push_back(g->n_leaf_groups);
            jobs.push_back(P2MJob{g->d_slot_groups, g->d_slot_entries, g->m, g->d_w, g->d_nx, g->d_ny, g->d_basis,
                                  g->basis_ord + 1, op->x, g->n, g->nslotcoef, op->nrhs, g->d_Mp});
            blocks.push_back(g->n_slot_groups);
        }
        launch_jobs(jobs, blocks, k_p2m_multi, 128, smem_p2m, s, "k_p2m_multi");
    }
    // M2M: pass k takes each geometry's parents at level D - 1 - k (down to its l0)
    for (int k = 0; k < max_up; ++k) {
        std::vector<XJob> jobs;
        std::vector<int> blocks;
        size_t smem = 0;
        for (const BatchOp* op : far) {
            lfmm_geometry_s* g = op->g;
            const TreeHost& t = g->tree;
            const int lp = t.D - 1 - k;
            if (lp < t.l0) continue;
            const XPass P = make_pass(g, lp + 1, 0, 0, op->nrhs);
            jobs.push_back(XJob{P, op->nrhs});
            blocks.push_back(xpass_fam_ctas(P.nq, P.fch) + P.nd * P.nch);
            smem = std::max(smem, xpass_smem(0, P.pS, P.pD, P.w));
        }
        raise_smem_limit((const void*)k_translate_multi, smem, "translate smem");
        launch_jobs(jobs, blocks, k_translate_multi, 128, smem, s, "k_translate_multi (M2M)");
    }
    {   // M2L of every level, then the reductions of split items
        std::vector<M2LJob> jobs;
        std::vector<int> blocks, rblocks;
        for (const BatchOp* op : far) {
            lfmm_geometry_s* g = op->g;
            const int D = g->tree.D;
            jobs.push_back(M2LJob{g->d_m2l_items, g->d_m2l_reds, g->d_m2l_ents, g->d_box_level, g->d_p_level,
                                  g->d_slot_of, g->d_coef_off, g->d_slot_coef, g->d_m2lf_off, g->d_m2lf, g->d_m2lr,
                                  op->nrhs, g->n_m2l_parts, g->ncoef, g->nslotcoef, g->d_M, g->d_Mp, g->d_L, g->d_Lp,
                                  g->d_m2l_part});
            blocks.push_back(g->m2l_item_level_start[D + 1]);
            rblocks.push_back(g->m2l_red_level_start[D + 1]);
        }
        launch_jobs(jobs, blocks, k_m2l_multi, 128, 0, s, "k_m2l_multi");
        launch_jobs(jobs, rblocks, k_m2l_reduce_multi, 64, 0, s, "k_m2l_reduce_multi");
    }
    // L2L: pass k takes each geometry's children at level l0 + 1 + k
    for (int k = 0; k < max_dn; ++k) {
        std::vector<XJob> jobs;
        std::vector<int> blocks;
        size_t smem = 0;
        for (const BatchOp* op : far) {
            lfmm_geometry_s* g = op->g;
            const TreeHost& t = g->tree;
            const int l = t.l0 + 1 + k;
            if (l > t.D) continue;
            const XPass P = make_pass(g, l, 1, 1, op->nrhs);
            jobs.push_back(XJob{P, op->nrhs});
            blocks.push_back(xpass_fam_ctas(P.nq, P.fch) + P.nd * P.nch);
            smem = std::max(smem, xpass_smem(1, P.pS, P.pD, P.w));
        }
        raise_smem_limit((const void*)k_translate_multi, smem, "translate smem");
        launch_jobs(jobs, blocks, k_translate_multi, 128, smem, s, "k_translate_multi (L2L)");
    }
    // L2P after the near field, which adds into the same y
    if (before_l2p) cuda_check(cudaStreamWaitEvent(s, before_l2p, 0), "wait for the near field");
    // the leaves about cell centres, then (a second launch: both add into the same points
    // of y) the straddling leaves about their reaction centres, as each geometry's own launches
    for (int slots = 0; slots < 2; ++slots) {
        std::vector<L2PJob> jobs;
        std::vector<int> blocks;
        for (const BatchOp* op : far) {
            lfmm_geometry_s* g = op->g;
            if (slots == 0) {
                jobs.push_back(L2PJob{g->d_leaf_groups, g->d_leaf_entries, g->d_basis, g->basis_ord + 1, g->n,
                                      g->ncoef, op->nrhs, g->d_L, op->y});
                blocks.push_back(g->n_leaf_groups);
            } else {
                jobs.push_back(L2PJob{g->d_slot_groups, g->d_slot_leaf_entries, g->d_basis, g->basis_ord + 1, g->n,
                                      g->nslotcoef, op->nrhs, g->d_Lp, op->y});
                blocks.push_back(g->n_slot_groups);
            }
        }
        launch_jobs(jobs, blocks, k_l2p_multi, 128, smem_l2p, s, "k_l2p_multi");
    }
}

// Schedule of the M2L work items chosen by measurement on this geometry: the cap
// on the work of one item (entries x output coefficients; heavier (box, chunk)s
// are split and their parts reduced) and whether an unsplit box with a narrow
// coefficient row gets one item for all of its coefficients.  Each candidate's
// FP64 M2L (items plus reductions) runs twice untimed and three times timed with
// CUDA events on the calling thread's stream, on zeroed expansions (the time of
// the FP64 pipe does not depend on the values), and the fastest is kept.  The
// schedule changes only the order in which the parts of a split sum are added.
void fmm_autotune(lfmm_geometry_s* g) {
    TreeHost& t = g->tree;
    if (t.l0 > t.D || g->n_m2l_items == 0) return;
    set_smem_limits();
    cudaStream_t s = cudaStreamPerThread;
    ensure_coef(g, 1);
    cuda_check(cudaMemsetAsync(g->d_M, 0, sizeof(cd) * std::max<int64_t>(g->ncoef, 1), s), "tune memset");
    cuda_check(cudaMemsetAsync(g->d_Mp, 0, sizeof(cd) * std::max<int64_t>(g->nslotcoef, 1), s), "tune memset");
    const int64_t launches = g->n_launches;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cuda_check(cudaEventCreate(&e0), "event");
    cuda_check(cudaEventCreate(&e1), "event");
    const int works[] = {1024, 2048, 4096, 8192};
    int best_work = g->m2l_item_work, best_wide = g->m2l_wide;
    double best = 1e300, dflt = 0.0;
    for (int wide = 1; wide >= 0; --wide) {
        for (int work : works) {
            make_m2l_items(g, work, wide);
            const int n64 = g->n_m2l_items, r64 = g->m2l_red_level_start[t.D + 2];
            for (int r = 0; r < 2; ++r) launch_m2l64(g, 1, n64, r64, s);
            cuda_check(cudaEventRecord(e0, s), "event");
            for (int r = 0; r < 3; ++r) launch_m2l64(g, 1, n64, r64, s);
            cuda_check(cudaEventRecord(e1, s), "event");
            cuda_check(cudaEventSynchronize(e1), "tune sync");
            float ms = 0.f;
            cuda_check(cudaEventElapsedTime(&ms, e0, e1), "event");
            const double per = ms / 3.0;
            if (work == M2L_ITEM_WORK && wide == 1) dflt = per;
            if (per < best) { best = per; best_work = work; best_wide = wide; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    make_m2l_items(g, best_work, best_wide);
    cuda_check(cudaStreamSynchronize(s), "tune");
    g->n_launches = launches;
    g->tune_ms_default = dflt;
    g->tune_ms_best = best;
}

}  // namespace lfmm
