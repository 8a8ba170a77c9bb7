// lfmm_internal.h -- host-side structures shared by the library's translation units.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lfmm.h"
#include "devmath.cuh"

namespace lfmm {

// A non-zero reaction component (Sec. 3.1, remark on zero components):
// matvec sources in layer ls (the Green's function's field layer) reached by a
// wave arriving up (a = 0) or down (a = 1); matvec targets in layer lt (the
// Green's function's source layer) left by a wave going up (b = 0) or down (b = 1).
struct Component {
    int ls, a, lt, b;
    double Hc;   // thickness of the layers the wave must cross (part of the effective distance)
};

struct TreeHost {
    // root square and depth
    double x0 = 0, y0 = 0, W = 1;
    int D = 0, l0 = 0, nbox = 0;
    std::vector<int> p_level;          // expansion order per level
    std::vector<int> perm;             // sorted position -> input index
    std::vector<int> layer_sorted;     // layer of the sorted points
    // boxes, ordered by (level, layer, Morton)
    std::vector<int> level_start;      // D+2 entries
    std::vector<int> box_level, box_layer, box_ix, box_iy, box_begin, box_end, box_parent;
    std::vector<int> child_begin, child_end;
    std::vector<Component> comps;
    // free-space lists (same layer): M2L (V) for every box, near (U) for leaves; CSR over boxes
    std::vector<int> vfree_ptr, vfree_idx, ufree_ptr, ufree_idx;
    // reaction lists: CSR over target boxes, entries (source box, component)
    std::vector<int> vreact_ptr, vreact_idx, vreact_comp;
    std::vector<int> ureact_ptr, ureact_idx, ureact_comp;

    double width(int l) const { return W / (double)(1u << l); }
    double cx(int b) const { return x0 + (box_ix[b] + 0.5) * width(box_level[b]); }
    double cy(int b) const { return y0 + (box_iy[b] + 0.5) * width(box_level[b]); }
};

// Builds the quadtree and all interaction lists on the host (tree.cpp: the reference
// statement of the tree definition, run by the CPU tests).  Throws std::runtime_error
// on invalid input.
void build_tree(TreeHost& t, const std::vector<double>& px, const std::vector<double>& py,
                const std::vector<int>& layer, const MediumDev& med, int p, int leaf_size);
// The same tree and lists built on the GPU from device arrays of the input points and
// their layers (tree_gpu.cu), equal to build_tree's bit for bit; the library builds every
// geometry's tree this way.
void build_tree_gpu(TreeHost& t, const double* d_px, const double* d_py, const int* d_layer, int64_t n,
                    const MediumDev& med, int p, int leaf_size);

// End of the real-axis stretch of the moment tables' contour, just past the largest
// branch point (the M2L table rule and the tree's admissibility test share it).
inline double table_detour_end(const MediumDev& m) { return m.kmax + 0.75; }
// Largest admitted log-growth of a column-separated reaction pair's table integrand
// (tree.cpp, reaction lists).
constexpr double REACT_COND_EXP = 16.0;

double comp_extra_thickness(const MediumDev& m, int ls, int a, int lt, int b);
double src_height(const MediumDev& m, int ls, int a, double y);
double tgt_height(const MediumDev& m, int lt, int b, double y);
double clipped_height(double yif, bool above, double lo, double hi);
double src_height_box(const MediumDev& m, int ls, int a, double lo, double hi);
double tgt_height_box(const MediumDev& m, int lt, int b, double lo, double hi);

}  // namespace lfmm
