// tree_harness.cpp -- runs the library's host tree builder (csrc/tree.cpp) on points
// read from a file and writes the tree and all interaction lists, so that a CPU test
// can compare them with the oracle's tree bit for bit at full workload sizes.
//
// Input (little-endian): int32 n, nl, p, leaf; float64 yint[nl-1], k[nl], eta[nl];
// float64 px[n], py[n]; int32 layer[n].
// Output: float64 x0, y0, W; int32 D, l0, ncomp, comps[4 ncomp]; then the int32
// arrays perm, layer_sorted, p_level, box_level, box_layer, box_ix, box_iy,
// box_begin, box_end, box_parent, vfree_ptr, vfree_idx, ufree_ptr, ufree_idx,
// vreact_ptr, vreact_idx, vreact_comp, ureact_ptr, ureact_idx, ureact_comp, each as
// int64 length followed by its values.
#include <algorithm>
#include <cstdio>
#include <cstdint>
#include <exception>
#include <vector>

#include "lfmm_internal.h"

template <class T>
static bool read_n(FILE* f, T* v, size_t n) {
    return std::fread(v, sizeof(T), n, f) == n;
}

template <class T>
static void write_n(FILE* f, const T* v, size_t n) {
    std::fwrite(v, sizeof(T), n, f);
}

static void write_array(FILE* f, const std::vector<int>& a) {
    const int64_t n = (int64_t)a.size();
    write_n(f, &n, 1);
    write_n(f, a.data(), a.size());
}

int main(int argc, char** argv) {
    if (argc != 3) {
        std::fprintf(stderr, "usage: tree_harness <input> <output>\n");
        return 2;
    }
    FILE* in = std::fopen(argv[1], "rb");
    if (!in) return 2;
    int32_t hdr[4];
    if (!read_n(in, hdr, 4)) return 2;
    const int n = hdr[0], nl = hdr[1], p = hdr[2], leaf = hdr[3];
    if (n < 1 || nl < 1 || nl > LFMM_MAXLAY) return 2;
    MediumDev m{};
    m.nl = nl;
    if (!read_n(in, m.yint, (size_t)(nl - 1)) || !read_n(in, m.k, (size_t)nl) || !read_n(in, m.eta, (size_t)nl))
        return 2;
    m.kmax = 0.0;
    for (int l = 0; l < nl; ++l) m.kmax = std::max(m.kmax, m.k[l]);
    std::vector<double> px(n), py(n);
    std::vector<int> layer(n);
    if (!read_n(in, px.data(), (size_t)n) || !read_n(in, py.data(), (size_t)n) ||
        !read_n(in, layer.data(), (size_t)n))
        return 2;
    std::fclose(in);

    lfmm::TreeHost t;
    try {
        lfmm::build_tree(t, px, py, layer, m, p, leaf);
    } catch (const std::exception& e) {
        std::fprintf(stderr, "build_tree: %s\n", e.what());
        return 3;
    }
    FILE* out = std::fopen(argv[2], "wb");
    if (!out) return 2;
    const double geo[3] = {t.x0, t.y0, t.W};
    write_n(out, geo, 3);
    const int32_t ints[3] = {t.D, t.l0, (int32_t)t.comps.size()};
    write_n(out, ints, 3);
    for (const auto& c : t.comps) {
        const int32_t cc[4] = {c.ls, c.a, c.lt, c.b};
        write_n(out, cc, 4);
    }
    for (const auto* a : {&t.perm, &t.layer_sorted, &t.p_level, &t.box_level, &t.box_layer, &t.box_ix, &t.box_iy,
                          &t.box_begin, &t.box_end, &t.box_parent, &t.vfree_ptr, &t.vfree_idx, &t.ufree_ptr,
                          &t.ufree_idx, &t.vreact_ptr, &t.vreact_idx, &t.vreact_comp, &t.ureact_ptr, &t.ureact_idx,
                          &t.ureact_comp})
        write_array(out, *a);
    std::fclose(out);
    return 0;
}
