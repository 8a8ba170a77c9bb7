// tree.cpp -- quadtree, layer boxes and interaction lists (host, C++).
//
// The paper runs its FMM on "the adaptive tree structure" without giving its
// parameters (Sec. 4.1); the definition implemented here is:
//  * root square around the bounding box of all points, side
//    W = max(extent) * (1 + 2^-10); coordinates quantised once to 20 bits;
//  * one box set per layer (points keep the layer of their height), all
//    layers sharing the root square and one depth D: the smallest level at
//    which no cell of any layer holds more than leaf_size points;
//  * points ordered by (layer, Morton key at level D, input index), boxes by
//    (level, layer, Morton key);
//  * expansion order per level p_l = max(p, ceil(kR + 9 (kR)^(1/3))),
//    kR = k_max w_l / sqrt(2); expansions are used from the first level
//    l0 >= 2 whose order is at most 80;
//  * free-space lists per layer (candidates = children of the parent's near
//    list; near = touching cells), and one set of lists per non-zero reaction
//    component, with the near/far decision taken in the image frame of the
//    component: horizontal cell offset, and vertical offset
//    D = h_*(S) + h_star(T) + H_c (the effective transmission distance of
//    Sec. 3.2 between the reaction expansion centres: cell centres, moved for
//    cells that straddle the interface to the middle of the part of the cell
//    on the layer's side).  A pair is far if D >= 2 w_l, or if the column
//    offset is at least 2 while |k_y(T')| (w_l - D) <= 16, T' = k_max + 0.75
//    the end of the moment tables' real-axis stretch, k_y for the smaller of
//    the two layers' wavenumbers: on that stretch the table integrand grows
//    like exp(|k_y| (w - D)) (the expansions' vertical extent, up to w / 2 on
//    each side, against the effective distance), and beyond exp(16) the
//    cancellation in the table costs accuracy (up to 3e-5 of an entry in the
//    four-layer medium k = 6, 10, 8, 12, wide-band cells with D << w).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <stdexcept>
#include <vector>

#include "lfmm_internal.h"

namespace lfmm {

static const int QBITS = 20;
static const int D_CAP = 18;
static const int P_CAP = 80;
static const int L0_MIN = 2;

static inline uint64_t morton2(uint32_t ix, uint32_t iy, int level) {
    uint64_t key = 0;
    for (int b = 0; b < level; ++b) {
        key |= (uint64_t)((ix >> b) & 1u) << (2 * b);
        key |= (uint64_t)((iy >> b) & 1u) << (2 * b + 1);
    }
    return key;
}

double comp_extra_thickness(const MediumDev& m, int ls, int a, int lt, int b) {
    auto H = [&](int q) { return m.yint[q - 1] - m.yint[q]; };
    if (ls == lt) return (a == b) ? H(ls) : 0.0;
    double h = 0.0;
    if (ls < lt) {
        for (int q = ls + 1; q < lt; ++q) h += H(q);
        if (a == 1) h += H(ls);
        if (b == 1) h += H(lt);
        return h;
    }
    for (int q = lt + 1; q < ls; ++q) h += H(q);
    if (a == 0) h += H(ls);
    if (b == 0) h += H(lt);
    return h;
}

double src_height(const MediumDev& m, int ls, int a, double y) {
    return (a == 0) ? (y - m.yint[ls]) : (m.yint[ls - 1] - y);
}

double tgt_height(const MediumDev& m, int lt, int b, double y) {
    return (b == 0) ? (m.yint[lt - 1] - y) : (y - m.yint[lt]);
}

// Height above (above = true) or below the interface y_if of the centre of the
// part of the cell [lo, hi] on the valid side: the reaction expansion centre of
// a box whose cell straddles the interface is moved there, so that every
// expansion centre lies on the side of its points.
double clipped_height(double yif, bool above, double lo, double hi) {
    if (above) return 0.5 * (std::max(lo, yif) + hi) - yif;
    return yif - 0.5 * (lo + std::min(hi, yif));
}

double src_height_box(const MediumDev& m, int ls, int a, double lo, double hi) {
    return (a == 0) ? clipped_height(m.yint[ls], true, lo, hi) : clipped_height(m.yint[ls - 1], false, lo, hi);
}

double tgt_height_box(const MediumDev& m, int lt, int b, double lo, double hi) {
    return (b == 0) ? clipped_height(m.yint[lt - 1], false, lo, hi) : clipped_height(m.yint[lt], true, lo, hi);
}

void build_tree(TreeHost& t, const std::vector<double>& px, const std::vector<double>& py,
                const std::vector<int>& layer, const MediumDev& med, int p, int leaf_size) {
    const int64_t n = (int64_t)px.size();
    if (n <= 0) throw std::runtime_error("build_tree: no points");
    double xmin = px[0], xmax = px[0], ymin = py[0], ymax = py[0];
    for (int64_t i = 1; i < n; ++i) {
        xmin = std::min(xmin, px[i]); xmax = std::max(xmax, px[i]);
        ymin = std::min(ymin, py[i]); ymax = std::max(ymax, py[i]);
    }
    double ext = std::max(xmax - xmin, ymax - ymin);
    double W = ext > 0 ? ext * (1.0 + 1.0 / 1024.0) : 1.0;
    double cx = 0.5 * (xmin + xmax), cy = 0.5 * (ymin + ymax);
    t.W = W;
    t.x0 = cx - 0.5 * W;
    t.y0 = cy - 0.5 * W;
    const double scale = (double)(1u << QBITS);
    const int64_t qmax = (1 << QBITS) - 1;
    std::vector<uint32_t> qx(n), qy(n);
    for (int64_t i = 0; i < n; ++i) {
        double fx = std::floor(((px[i] - t.x0) / W) * scale);
        double fy = std::floor(((py[i] - t.y0) / W) * scale);
        int64_t a = (int64_t)fx, b = (int64_t)fy;
        qx[i] = (uint32_t)std::min<int64_t>(std::max<int64_t>(a, 0), qmax);
        qy[i] = (uint32_t)std::min<int64_t>(std::max<int64_t>(b, 0), qmax);
    }
    // depth: smallest level with at most leaf_size points per (layer, cell)
    int D = D_CAP;
    {
        std::vector<uint64_t> keys(n);
        for (int l = 0; l <= D_CAP; ++l) {
            int sh = QBITS - l;
            for (int64_t i = 0; i < n; ++i)
                keys[i] = ((uint64_t)layer[i] << 56) | ((uint64_t)(qx[i] >> sh) << 28) | (uint64_t)(qy[i] >> sh);
            std::sort(keys.begin(), keys.end());
            int run = 1, worst = 1;
            for (int64_t i = 1; i < n; ++i) {
                run = (keys[i] == keys[i - 1]) ? run + 1 : 1;
                worst = std::max(worst, run);
            }
            if (worst <= leaf_size) { D = l; break; }
        }
    }
    t.D = D;
    t.p_level.assign(D + 1, p);
    for (int l = 0; l <= D; ++l) {
        double kr = med.kmax * (W / (double)(1u << l)) * 0.70710678118654752;
        int pl = (int)std::ceil(kr + 9.0 * std::pow(kr, 1.0 / 3.0));
        t.p_level[l] = std::max(p, pl);
    }
    t.l0 = D + 1;
    for (int l = L0_MIN; l <= D; ++l)
        if (t.p_level[l] <= P_CAP) { t.l0 = l; break; }

    // point order: (layer, Morton at level D, input index)
    {
        int sh = QBITS - D;
        std::vector<std::pair<uint64_t, int>> order(n);
        for (int64_t i = 0; i < n; ++i) {
            uint64_t key = ((uint64_t)layer[i] << 48) | morton2(qx[i] >> sh, qy[i] >> sh, D);
            order[i] = {key, (int)i};
        }
        std::sort(order.begin(), order.end());
        t.perm.resize(n);
        t.layer_sorted.resize(n);
        for (int64_t s = 0; s < n; ++s) {
            t.perm[s] = order[s].second;
            t.layer_sorted[s] = layer[order[s].second];
        }
    }
    // boxes, level by level
    t.level_start.clear();
    t.box_level.clear(); t.box_layer.clear(); t.box_ix.clear(); t.box_iy.clear();
    t.box_begin.clear(); t.box_end.clear(); t.box_parent.clear();
    for (int l = 0; l <= D; ++l) {
        t.level_start.push_back((int)t.box_level.size());
        int sh = QBITS - l;
        int prev_lay = -1;
        uint32_t prev_x = 0, prev_y = 0;
        int pbox = (l > 0) ? t.level_start[l - 1] : -1;  // monotone pointer into level l-1
        for (int64_t s = 0; s < n; ++s) {
            int i = t.perm[s];
            uint32_t cxq = qx[i] >> sh, cyq = qy[i] >> sh;
            int lay = layer[i];
            if (lay != prev_lay || cxq != prev_x || cyq != prev_y) {
                t.box_level.push_back(l);
                t.box_layer.push_back(lay);
                t.box_ix.push_back((int)cxq);
                t.box_iy.push_back((int)cyq);
                t.box_begin.push_back((int)s);
                t.box_end.push_back((int)s + 1);
                if (l > 0) {
                    while (!(t.box_begin[pbox] <= s && s < t.box_end[pbox])) ++pbox;
                    t.box_parent.push_back(pbox);
                } else {
                    t.box_parent.push_back(-1);
                }
                prev_lay = lay; prev_x = cxq; prev_y = cyq;
            } else {
                t.box_end.back() = (int)s + 1;
            }
        }
    }
    t.level_start.push_back((int)t.box_level.size());
    const int nb = (int)t.box_level.size();
    t.nbox = nb;
    t.child_begin.assign(nb, 0);
    t.child_end.assign(nb, 0);
    for (int b = 0; b < nb; ++b) {
        int pb = t.box_parent[b];
        if (pb < 0) continue;
        if (t.child_end[pb] == 0) t.child_begin[pb] = b;
        t.child_end[pb] = b + 1;
    }

    // free-space lists
    {
        std::vector<std::vector<int>> nearl(nb), vl(nb);
        for (int l = 0; l <= D; ++l) {
            for (int T = t.level_start[l]; T < t.level_start[l + 1]; ++T) {
                std::vector<int> cands;
                if (l == 0) {
                    cands.push_back(T);
                } else {
                    for (int S : nearl[t.box_parent[T]])
                        for (int c = t.child_begin[S]; c < t.child_end[S]; ++c) cands.push_back(c);
                }
                for (int S : cands) {
                    if (l < t.l0) { nearl[T].push_back(S); continue; }
                    if (std::abs(t.box_ix[S] - t.box_ix[T]) <= 1 && std::abs(t.box_iy[S] - t.box_iy[T]) <= 1)
                        nearl[T].push_back(S);
                    else
                        vl[T].push_back(S);
                }
            }
        }
        t.vfree_ptr.assign(nb + 1, 0);
        t.ufree_ptr.assign(nb + 1, 0);
        t.vfree_idx.clear(); t.ufree_idx.clear();
        for (int b = 0; b < nb; ++b) {
            for (int S : vl[b]) t.vfree_idx.push_back(S);
            if (t.box_level[b] == D) for (int S : nearl[b]) t.ufree_idx.push_back(S);
            t.vfree_ptr[b + 1] = (int)t.vfree_idx.size();
            t.ufree_ptr[b + 1] = (int)t.ufree_idx.size();
        }
    }

    // reaction components and their lists
    const int L = med.nl - 1;
    t.comps.clear();
    for (int ls = 0; ls <= L; ++ls)
        for (int a = 0; a < 2; ++a) {
            if (a == 0 && ls >= L) continue;
            if (a == 1 && ls <= 0) continue;
            for (int lt = 0; lt <= L; ++lt)
                for (int b = 0; b < 2; ++b) {
                    if (b == 0 && lt <= 0) continue;
                    if (b == 1 && lt >= L) continue;
                    Component c{ls, a, lt, b, comp_extra_thickness(med, ls, a, lt, b)};
                    t.comps.push_back(c);
                }
        }
    const int nc = (int)t.comps.size();
    std::vector<std::vector<std::pair<int, int>>> vr(nb), ur(nb);  // (comp, S)
    const double t_tab = table_detour_end(med);
    for (int c = 0; c < nc; ++c) {
        const Component& C = t.comps[c];
        const double kl = std::min(med.k[C.ls], med.k[C.lt]);
        const double ky_tab = std::sqrt(t_tab * t_tab - kl * kl);
        std::vector<std::vector<int>> nearl(nb);
        for (int l = 0; l <= D; ++l) {
            double w = t.width(l);
            for (int T = t.level_start[l]; T < t.level_start[l + 1]; ++T) {
                if (t.box_layer[T] != C.lt) continue;
                std::vector<int> cands;
                if (l == 0) {
                    for (int S = t.level_start[0]; S < t.level_start[1]; ++S)
                        if (t.box_layer[S] == C.ls) cands.push_back(S);
                } else {
                    for (int S : nearl[t.box_parent[T]])
                        for (int ch = t.child_begin[S]; ch < t.child_end[S]; ++ch) cands.push_back(ch);
                }
                for (int S : cands) {
                    if (l < t.l0) { nearl[T].push_back(S); continue; }
                    double loS = t.y0 + t.box_iy[S] * w, hiS = t.y0 + (t.box_iy[S] + 1) * w;
                    double loT = t.y0 + t.box_iy[T] * w, hiT = t.y0 + (t.box_iy[T] + 1) * w;
                    double Dc = (src_height_box(med, C.ls, C.a, loS, hiS) + tgt_height_box(med, C.lt, C.b, loT, hiT)) +
                                C.Hc;
                    bool far = (std::abs(t.box_ix[S] - t.box_ix[T]) >= 2 && ky_tab * (w - Dc) <= REACT_COND_EXP) ||
                               Dc >= 2.0 * w * (1.0 - 1e-9);
                    if (far) vr[T].push_back({c, S});
                    else nearl[T].push_back(S);
                }
                if (l == D)
                    for (int S : nearl[T]) ur[T].push_back({c, S});
            }
        }
    }
    t.vreact_ptr.assign(nb + 1, 0);
    t.ureact_ptr.assign(nb + 1, 0);
    t.vreact_idx.clear(); t.vreact_comp.clear(); t.ureact_idx.clear(); t.ureact_comp.clear();
    for (int b = 0; b < nb; ++b) {
        for (auto& e : vr[b]) { t.vreact_comp.push_back(e.first); t.vreact_idx.push_back(e.second); }
        for (auto& e : ur[b]) { t.ureact_comp.push_back(e.first); t.ureact_idx.push_back(e.second); }
        t.vreact_ptr[b + 1] = (int)t.vreact_idx.size();
        t.ureact_ptr[b + 1] = (int)t.ureact_idx.size();
    }
}

}  // namespace lfmm
