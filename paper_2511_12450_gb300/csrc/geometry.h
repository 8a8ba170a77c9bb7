// geometry.h -- the opaque handles behind the C ABI and the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <functional>
#include <mutex>
#include <cstdint>
#include <string>
#include <algorithm>
#include <vector>

#include "lfmm_internal.h"

struct lfmm_medium_s {
    MediumDev m;
    std::atomic<int> geometries{0};   // live geometries referencing this medium (built on any thread)
};

namespace lfmm {

// device buffer owned by a geometry
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
};

// Sommerfeld quadrature parameters shared by host and device (passed by value)
struct QuadRule {
    double T;          // end of the real-axis detour
    double kmin;       // smallest wavenumber of the medium (the first branch point on the detour)
    double es_v0;      // exp-sinh abscissae v0 + j hv, j = 0..nes-1
    double es_hv;
    int nes;           // nodes per ray
    int min_panels;    // minimum number of detour panels
    // rule of the M2L moment tables, whose integrands carry w^n factors up to
    // |n - m| = 2p: more detour panels (pS + pT more) and their own rays
    double tab_es_v0, tab_es_hv;
    int tab_nes;
    int tab_panel_mult;
    // end of the tables' detour, just past the largest branch point: the moments of
    // an expansion layer with k < k_max carry |w|^{-n} ~ (2 lambda / k)^n over its
    // evanescent range (k, T), which largely cancels, so a shorter real-axis
    // stretch keeps the rounding of the moments small
    double tab_T;
    double gl_x[8];    // 8-point Gauss-Legendre rule on [-1, 1]
    double gl_w[8];
};

// point range expanded about one centre (P2M / L2P)
struct ExpEntry {
    int beg, end, lay, p;
    double cx, cy;
    int64_t off;   // coefficient offset in the output/input array
    int64_t brow;  // row of the entry's first point in the stored expansion basis
};
// consecutive entries processed by one CTA (at most EXP_GROUP_PTS points and
// EXP_GROUP_ENTRIES entries, or a single larger entry)
#define EXP_GROUP_PTS 64
#define EXP_GROUP_ENTRIES 16
struct ExpGroup {
    int e0, e1;    // entry range
    int npts;      // points of the group
};
// M2M / L2L pass records (see k_translate)
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
// A parent cell and its children about cell centres: the quadrant form of M2M and
// L2L (k_translate).  Children are stored by quadrant (ix & 1) | ((iy & 1) << 1); the
// quadrant-3 child (+w/2, +w/2) carries the base vectors.  A child that also takes a
// straddling parent's reaction-centre local is an L2L destination of its own (dn_skip).
struct QuadX {
    int64_t par;          // parent's coefficient offset
    int64_t ch[4];        // children's coefficient offsets by quadrant (-1: no child)
    int64_t vup, vdn;     // base vectors of the family's layer and level (M2M; L2L reversed)
    int lay;              // the family's layer
    int dn_skip;          // bit q: the L2L of child q is a destination of its own
};
// M2L work: XT_W output coefficients of one target box over a range of its
// list entries; part >= 0 sends the partial sums to the reduction buffer.
#define XT_W 16
struct M2LItem {
    int box, chunk;
    int e0, e1;       // entry range (M2LEnt indices)
    int part;         // -1: write L directly; else partial-sum slot (always XT_W lanes)
    int w;            // output lanes per row: XT_W (chunks of XT_W coefficients) or 2p+1 (all of them)
};
// CTAs a block right-hand side's columns are split over in the translation and double-float
// M2L kernels (groups of four columns); one column keeps one CTA
inline int col_groups(int nrhs) { return nrhs <= 2 ? 1 : (nrhs + 3) / 4; }
// Lanes per output row for nco coefficients on a 128-thread CTA: chunks of XT_W
// lanes (8 slices of the sum), or one lane per coefficient with 128 / nco slices,
// whichever keeps more threads on an output (41 of 48 vs 123 of 128 at p = 20).
inline int lane_width(int nco) {
    if (nco > 128) return XT_W;
    const int chunks = (nco + XT_W - 1) / XT_W;
    const double u16 = (double)nco / (double)(XT_W * chunks);
    const double uf = (double)(nco * (128 / nco)) / 128.0;
    return (uf > u16 + 0.02) ? nco : XT_W;
}
// CTAs (4 warps) of a pass's families
__host__ __device__ inline int xpass_fam_ctas(int nq, int fch) { return (nq * fch + 3) / 4; }
// warps per family and rounds per warp: whole families per warp when there are enough
// of them to fill the GPU (16 warps per SM), else each family split over more warps
inline void xpass_fam_split(int nq, int pD, int* fch, int* fr) {
    const int rounds = (4 * (2 * pD + 1) + 31) / 32;
    const int want = nq > 0 ? (152 * 16 + nq - 1) / nq : 1;
    const int ch = std::max(1, std::min(rounds, want));
    *fr = (rounds + ch - 1) / ch;
    *fch = (rounds + *fr - 1) / *fr;
}

// one list entry of a target box
// M2L_FLIP: the table is that of the mirrored pair (offset -X), read with both
// indices reversed
enum { M2L_REACT = 1, M2L_SRC_SLOT = 2, M2L_A_DOWN = 4, M2L_B_DOWN = 8, M2L_FLIP = 16, M2L_DST_SHIFT = 5 };
struct M2LEnt {
    int64_t src;      // source coefficient offset (M, or Mp with M2L_SRC_SLOT)
    int64_t tab;      // free space: table id; reaction: offset of the moment table
    int flags;        // M2L_* bits; output array (0 = L, 1/2 = side-0/1 reaction centre) at M2L_DST_SHIFT
    int pad;
};
// a (box, chunk) whose entries were split: parts [part0, part0 + nparts)
struct M2LReduce {
    int box, chunk, part0, nparts;
};
struct MixedState;

// reaction M2L table key (built on the host, evaluated on the device)
struct ReactKey {
    int comp, level, pS, pT;   // component, level, orders of source/target expansions
    double X, hS, hT, D;       // x_S - x_T, source-side and target-side heights, effective distance
    int64_t off;               // offset of the (2pT+1) x (2pS+1) table, column-major: (m, n) at n (2pT+1) + m
};

}  // namespace lfmm

namespace lfmm {
enum Stage { ST_P2M = 0, ST_M2M, ST_M2L, ST_L2L, ST_L2P, ST_NEAR, ST_GATHER, ST_SCATTER, ST_COUNT };
struct StageProfiler {
    bool on = false;
    cudaEvent_t ev[2 * ST_COUNT] = {};
    bool armed[ST_COUNT] = {};
    double ms[ST_COUNT] = {};
    double cnt[ST_COUNT] = {};
};
}  // namespace lfmm

struct lfmm_geometry_s {
    lfmm::StageProfiler prof;
    int64_t n_launches = 0;           // kernels this geometry's matvec path has launched (host count)
    lfmm_medium_s* med = nullptr;
    MediumDev m;
    int64_t n = 0;
    // points with input index >= n_src are field points (weight 0) of a field
    // geometry built by lfmm_eval_field; n_src = n for a geometry of elements only
    int64_t n_src = 0;
    int p = 20, leaf_size = 64;
    lfmm::TreeHost tree;
    lfmm::QuadRule quad;
    std::vector<double> hx, hy, hw;   // sorted-order host copies
    std::vector<double> hnx, hny;     // sorted-order normals (combined field only)
    int nleaf = 0, leaf0 = 0;         // leaves are boxes [leaf0, leaf0 + nleaf)

    // sorted-order point data
    double *d_x = nullptr, *d_y = nullptr, *d_w = nullptr;
    bool combined = false;                   // combined-field operator (LFMM_COMBINED_FIELD)
    bool m2l_simt = false;                   // this call: FP32 M2L on the SIMT kernel only (LFMM_SIMT_M2L)
    cudaStream_t side = nullptr;             // near field beside the far field (apply_operator_sorted)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double *d_nx = nullptr, *d_ny = nullptr; // outward unit normals (sorted order), combined field only
    int *d_layer = nullptr, *d_perm = nullptr;
    // boxes
    int *d_box_begin = nullptr, *d_box_end = nullptr, *d_box_layer = nullptr, *d_box_level = nullptr;
    double *d_box_cx = nullptr, *d_box_cy = nullptr;
    int *d_box_ix = nullptr, *d_box_iy = nullptr, *d_box_parent = nullptr;
    int *d_child_begin = nullptr, *d_child_end = nullptr;
    int64_t *d_coef_off = nullptr;    // per box offset into M / L
    int64_t ncoef = 0;
    cd *d_M = nullptr, *d_L = nullptr;   // [coef_cols][ncoef]
    int coef_cols = 0;
    // reaction expansion centres moved off the cell centre (cells straddling an interface):
    // one slot per (box, side), side 0 = the layer's bottom interface, 1 = its top interface
    int n_slots = 0;
    int64_t nslotcoef = 0;
    int *d_slot_of = nullptr;          // [2 * nbox] slot index or -1
    int64_t *d_slot_coef = nullptr;
    cd *d_Mp = nullptr, *d_Lp = nullptr;   // [coef_cols][nslotcoef]
    // P2M/L2P work lists (leaves about cell centres; straddling boxes/leaves about reaction centres)
    int n_leaf_entries = 0, n_slot_entries = 0, n_slot_leaf_entries = 0;
    lfmm::ExpEntry *d_leaf_entries = nullptr, *d_slot_entries = nullptr, *d_slot_leaf_entries = nullptr;
    lfmm::ExpGroup *d_leaf_groups = nullptr, *d_slot_groups = nullptr;   // P2M / L2P work groups
    // J_n(k rho) e^{i n theta}, n = 0..basis_ord, one row per (entry, point): leaf entries at
    // rows 0..n-1 (the point's index), straddling leaves' reaction-centre entries after them
    cd* d_basis = nullptr;
    int basis_ord = 0;
    int n_leaf_groups = 0, n_slot_groups = 0, group_max_pts = 1, group_max_ent = 1;
    // M2M (up) and L2L (down) passes: per level, a range of destinations
    // (cells and reaction centres) with their sources and translation vectors
    std::vector<int> up_begin, up_end, dn_begin, dn_end;
    // parent/child cell families per child level (q_begin[l]..q_end[l]: parents at l - 1)
    std::vector<int> q_begin, q_end;
    lfmm::QuadX* d_qx = nullptr;
    std::vector<lfmm::QuadX> qx_host;
    std::vector<int64_t> qvec_host;   // base vector per ((layer nlev + child level) 2 + down), -1: none
    lfmm::XDst* d_xdst = nullptr;
    lfmm::XSrc* d_xsrc = nullptr;
    cd* d_xvec = nullptr;
    std::vector<lfmm::XDst> xdst_host;
    std::vector<lfmm::XSrc> xsrc_host;
    std::vector<int> xd_layer_host;
    // near field: block-sparse rows over target leaves
    int *d_nb_ptr = nullptr;          // nleaf + 1
    int *d_nb_src = nullptr;          // source leaf (box id) per block
    int64_t *d_nb_off = nullptr;      // value offset per block
    cd *d_nb_val = nullptr;           // blocks stored column-major (source index major)
    int64_t nb_nnz = 0;
    int n_blocks = 0;
    // a target leaf's blocks lie one after another: one nT x nJ column-major matrix per leaf
    int64_t *d_nl_off = nullptr;      // per leaf: offset of its first block
    int *d_nl_jptr = nullptr;         // per leaf: column range
    int *d_nl_j = nullptr;            // per column: sorted source position
    std::vector<int> nb_ptr_host, nb_src_host;
    std::vector<int64_t> nb_off_host;
    std::vector<unsigned char> nb_react_host;   // 1: the block holds reaction entries
    // precision form of the near field (built on its first use): blocks without reaction
    // entries in complex64 (self terms moved to an FP64 diagonal), the others in FP64
    bool near32_ready = false;
    float2 *d_nv32 = nullptr;
    int64_t *d_nl_off32 = nullptr;
    int *d_nl_jptr32 = nullptr, *d_nl_j32 = nullptr;
    cd *d_nv64r = nullptr;
    int64_t *d_nl_off64r = nullptr;
    int *d_nl_jptr64r = nullptr, *d_nl_j64r = nullptr;
    cd *d_ndiag = nullptr;
    int64_t near32_nnz = 0, near64r_nnz = 0;
    float2 *d_near_x32 = nullptr;     // x rounded to complex64 for the FP32 near-field products
    int64_t near_x32_cap = 0;
    // translation tables
    int *d_p_level = nullptr;
    cd *d_m2lf = nullptr;             // free-space M2L: per (layer, level, offset) Toeplitz vectors
    int64_t m2lf_len = 0;             // its length (complex values)
    int64_t *d_m2lf_off = nullptr;
    int *d_vf_ptr = nullptr, *d_vf_src = nullptr, *d_vf_tab = nullptr;   // free V lists with table ids
    lfmm::M2LItem* d_m2l_items = nullptr;   // coarse levels first
    lfmm::M2LEnt* d_m2l_ents = nullptr;     // entry descriptors, per target box in list order
    lfmm::M2LReduce* d_m2l_reds = nullptr;  // split (box, chunk)s
    int n_m2l_items = 0, n_m2l_parts = 0;
    std::vector<int> m2l_item_level_start;  // [nlev + 2]: first item of each level (levels > D: the end)
    std::vector<int> m2l_red_level_start;   // same for the reductions
    cd* d_m2l_part = nullptr;               // partial sums [cols][n_m2l_parts][3][XT_W]
    int m2l_part_cols = 0;
    std::vector<int> vf_ptr_host, vf_src_host, vf_tab_host, slot_of_host;
    std::vector<int> m2l_ent_ptr_host;      // entry range per target box
    int m2l_item_work = 0, m2l_wide = 1;    // schedule of the items (see make_m2l_items)
    double tune_ms_default = 0.0, tune_ms_best = 0.0;   // M2L launch times measured by the autotuner
    cd *d_m2lr = nullptr;             // reaction M2L tables
    int *d_vr_ptr = nullptr, *d_vr_src = nullptr, *d_vr_key = nullptr, *d_vr_comp = nullptr;
    lfmm::ReactKey* d_rkeys = nullptr;
    // host copies kept for the precision form's tables
    std::vector<lfmm::ReactKey> rkeys_host;
    std::vector<int> rkey_lay_s, rkey_lay_t;       // layers of the source / target boxes of each key
    std::vector<int> ftab_lay, ftab_lev;           // layer and level of each free-space M2L table
    std::vector<int> slot_box_host;
    std::vector<int64_t> box_coef_off_host;
    std::vector<int64_t> slot_coef_host;
    // precision form (FP32 M2L with scaled coefficients), built on first use
    lfmm::MixedState* mixed = nullptr;
    int n_rkeys = 0;
    int* d_comp = nullptr;            // 4 ints per component
    // level bookkeeping for launches
    std::vector<int> level_start;
    // scratch
    cd *d_xs = nullptr, *d_ys = nullptr;   // sorted-order input/output (n * nrhs_cap)
    int nrhs_cap = 0;
    cd *d_hostbuf_x = nullptr, *d_hostbuf_y = nullptr;  // staging for host-pointer calls
    size_t hostbuf_cap = 0;
    // preconditioner (restricted overlapping DD, Sec. 4.2)
    int *d_pc_ptr = nullptr;          // per leaf: offset of its gather list
    int pc_qmax = 0;                  // largest gather list
    int *d_pc_idx = nullptr;          // gather indices (sorted positions)
    int64_t *d_pc_woff = nullptr;     // per leaf: offset of its (n_own x q) row block
    cd *d_pc_W = nullptr;
    int *pc_own_first = nullptr, *pc_own_cnt = nullptr;
    bool pc_ready = false;
    double setup_seconds = 0.0;
    double setup_phase[3] = {0.0, 0.0, 0.0};   // seconds: tree and lists, near field, far field (tables, plans)
    double table_cmacs[2] = {0.0, 0.0};        // complex multiply-adds of the moment tables: cross-layer, same-layer
    int64_t m2lr_len = 0, pc_w_len = 0;         // entries of the reaction tables and of the preconditioner's W
    std::vector<void*> allocs;        // everything cudaMalloc'ed for this geometry
    // held by every call that applies the operator or the preconditioner to vectors
    // (matvec, the allocation-free matvec, precondition, solve, right-hand side, field):
    // calls on one geometry run one after another even if a caller does not serialise them
    std::mutex call_mu;
};

namespace lfmm {

// error helpers (api.cu)
void set_error(const std::string& msg);
struct CudaError {
    std::string msg;
};
struct TimeoutError {   // a bounded device wait gave up (LFMM_ERR_TIMEOUT)
    std::string msg;
};
struct ArgError {       // an invalid argument (LFMM_ERR_INVALID_ARG)
    std::string msg;
};
struct QuadratureError { // a stored kernel value or translation table is not finite (LFMM_ERR_QUADRATURE)
    std::string msg;
};
struct InterfaceError { // a point on an interface (LFMM_ERR_NODE_ON_INTERFACE)
    std::string msg;
};
// Runs f and maps every exception to the entry points' status codes; a failed call
// also clears the thread's last CUDA error (api.cu).
lfmm_status guarded_call(const std::function<lfmm_status()>& f);
void cuda_check(cudaError_t e, const char* what);
// Device memory of a geometry.  Allocations are stream-ordered on the calling
// thread's default stream so that building or releasing one geometry does not
// synchronise the device (other geometries' work keeps running).
// dev_alloc_ready: a work buffer, ready for use on any stream when it returns.
inline void* dev_alloc_ready(size_t bytes, const char* what) {
    void* p = nullptr;
    cuda_check(cudaMallocAsync(&p, bytes, cudaStreamPerThread), what);
    cuda_check(cudaStreamSynchronize(cudaStreamPerThread), what);
    return p;
}
// dev_release_now: a work buffer being replaced by a larger one; work queued on
// any stream may still read it, so the device is synchronised first (rare).
inline void dev_release_now(void* p) {
    if (p) { cudaDeviceSynchronize(); cudaFree(p); }
}
// dev_release: release at destroy; the caller guarantees that no work using the
// geometry is in flight (every stream it passed has been synchronised).
inline void dev_release(void* p) {
    if (p) cudaFreeAsync(p, cudaStreamPerThread);
}
template <class T>
T* dalloc(lfmm_geometry_s* g, size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    // stream-ordered: no device-wide synchronisation, so work of other geometries keeps
    // running while this one is built (the build synchronises its own stream at the end)
    cuda_check(cudaMallocAsync(&p, count * sizeof(T), cudaStreamPerThread), "cudaMallocAsync");
    g->allocs.push_back(p);
    return (T*)p;
}
template <class T>
T* dupload(lfmm_geometry_s* g, const std::vector<T>& v) {
    T* p = dalloc<T>(g, v.size());
    // from pageable memory the call returns once the source has been staged
    if (!v.empty())
        cuda_check(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, cudaStreamPerThread),
                   "upload");
    return p;
}

// near field (near.cu)
void near_build(lfmm_geometry_s* g);
void near_apply(lfmm_geometry_s* g, const cd* x_sorted, cd* y_sorted, int nrhs, cudaStream_t s, bool mixed = false);
// FMM far field (fmm.cu)
void fmm_build(lfmm_geometry_s* g);
void fmm_apply(lfmm_geometry_s* g, const cd* x_sorted, cd* y_sorted, int nrhs, cudaStream_t s, bool mixed = false,
               cudaEvent_t before_l2p = nullptr);
void fmm_autotune(lfmm_geometry_s* g);
// One operator product per geometry, several geometries in shared launches: every stage
// (near field, P2M, each M2M pass, M2L and its reductions, each L2L pass, L2P) is one
// launch whose blocks cover all the geometries' work (batch.cu helpers below).  FP64
// operator; x and y in each geometry's sorted order.
struct BatchOp {
    lfmm_geometry_s* g;
    const cd* x;
    cd* y;
    int nrhs;
};
// Device copies of per-launch job tables, released on the stream after use.
struct JobTables {
    std::vector<unsigned char> host;
    size_t add(const void* p, size_t bytes) {
        const size_t o = (host.size() + 15) & ~(size_t)15;
        host.resize(o + bytes);
        std::memcpy(host.data() + o, p, bytes);
        return o;
    }
    unsigned char* dev = nullptr;
    void upload(cudaStream_t s);
    void release(cudaStream_t s);
    template <class T>
    const T* at(size_t o) const { return (const T*)(dev + o); }
};
void fmm_apply_batch(const std::vector<BatchOp>& ops, cudaStream_t s, cudaEvent_t before_l2p);
void near_apply_batch(const std::vector<BatchOp>& ops, cudaStream_t s);
void apply_operator_batch_sorted(const std::vector<BatchOp>& ops, cudaStream_t s);
// Raise (never lower) a kernel's dynamic shared-memory limit on the current device.
// The attribute is process-wide, shared by every geometry and thread, so a
// geometry that needs less must not undo what another one was granted.
void raise_smem_limit(const void* func, size_t bytes, const char* what);
// precision form: M2L in FP32 on scaled expansions (mixed.cu)
void mixed_setup(lfmm_geometry_s* g, int nrhs);                       // tables, scales, FP32 buffers
void mixed_p2m(lfmm_geometry_s* g, const cd* x_sorted, int nrhs, cudaStream_t s);
void mixed_m2m(lfmm_geometry_s* g, int parent_level, int nrhs, cudaStream_t s);
void mixed_m_to64(lfmm_geometry_s* g, int level, int nrhs, cudaStream_t s);   // FP32 multipoles -> FP64
void mixed_m2l(lfmm_geometry_s* g, int nrhs, int min_level, cudaStream_t s);
// the M2L work items [0, n_items) (the levels below the first FP32 level) in double-float;
// writes the FP64 locals and partial sums (the caller adds the reductions)
bool mixed_coarse_df(lfmm_geometry_s* g);
// first FP32 level of the precision form, whether its coarser levels' M2L runs in
// double-float (1), in FP64 (0), or is not set up yet (-1: no precision-form call so far), and
// the log10 magnitudes that decided it (largest free-space and reaction table component, largest
// scaled multipole basis value)
void mixed_info(lfmm_geometry_s* g, int* lm, int* df, double* range);
void mixed_m2l_coarse(lfmm_geometry_s* g, int nrhs, int n_items, cudaStream_t s);
void mixed_l_add(lfmm_geometry_s* g, int level, int nrhs, cudaStream_t s);    // FP64 locals += into FP32
void mixed_l2l(lfmm_geometry_s* g, int child_level, int nrhs, cudaStream_t s);
void mixed_l2p(lfmm_geometry_s* g, cd* y_sorted, int nrhs, cudaStream_t s);
int mixed_level(lfmm_geometry_s* g);   // first level whose M2L runs in FP32
void mixed_destroy(lfmm_geometry_s* g);
// Throws TimeoutError, once, if a bounded wait of the tensor-core M2L gave up in work
// this geometry's host copy of the status has seen (copied after every launch; current
// once the launching stream has been synchronised).  Clears the status.
void mixed_check_waits(lfmm_geometry_s* g);
void fmm_free(lfmm_geometry_s* g);   // per-nrhs coefficient buffers
// permutation helpers and the full operator (solver.cu)
void gather_sorted(lfmm_geometry_s* g, const cd* x_in, cd* x_sorted, int nrhs, cudaStream_t s);
void scatter_sorted(lfmm_geometry_s* g, const cd* y_sorted, cd* y_out, int nrhs, cudaStream_t s);
void gather_sorted_c64(lfmm_geometry_s* g, const float2* x_in, cd* x_sorted, int nrhs, cudaStream_t s);
void scatter_sorted_c64(lfmm_geometry_s* g, const cd* y_sorted, float2* y_out, int nrhs, cudaStream_t s);
void round_to_c64(const cd* in, float2* out, int64_t n, cudaStream_t s);
void apply_operator_sorted(lfmm_geometry_s* g, const cd* x_sorted, cd* y_sorted, int nrhs, cudaStream_t s,
                           bool mixed = false);
void precond_build(lfmm_geometry_s* g);
// non-finite entries of the stored near field, free-space and reaction tables and preconditioner
void count_nonfinite(lfmm_geometry_s* g, double out[4]);
// per reaction table: component, level, order, X, hS, hT, D, non-finite entries
void react_key_report(lfmm_geometry_s* g, std::vector<double>& out);
// lockstep solves of the serving loop (solver.cu): create on the request's stream (builds
// the preconditioner, gathers b from input order), then begin, rounds and finish on the
// engine's stream; destroy releases everything
struct BatchSolve;
BatchSolve* batch_solve_create(lfmm_geometry_s* g, const cd* b_in, double tol, int maxit, bool pre, int precision,
                               cudaStream_t s);
void batch_solve_begin(BatchSolve* S, cudaStream_t s);
void batch_solve_round(const std::vector<BatchSolve*>& all, cudaStream_t s);
bool batch_solve_done(const BatchSolve* S);
void batch_solve_finish(BatchSolve* S, cd* x_out, lfmm_gmres_info* info, cudaStream_t s);
void batch_solve_destroy(BatchSolve* S, cudaStream_t s);
int gmres_sorted(lfmm_geometry_s* g, const cd* b, cd* x, int nrhs, double tol, int maxit, bool pre,
                 cudaStream_t s, lfmm_gmres_info* info, int precision = 0, int restart = 0);
void precond_apply_sorted(lfmm_geometry_s* g, const cd* v_sorted, cd* z_sorted, cudaStream_t s);
void rhs_plane_wave_sorted(lfmm_geometry_s* g, int nrhs, const double* angles_host, cd* b_sorted, cudaStream_t s);
// scattered field through a field geometry (api.cu builds it): x = [Phi; 0] per column,
// u = (field-point rows of K x) / eta of each field point's layer
void field_pack(const void* phi, bool c64, int64_t n, int64_t m, int nrhs, cd* x, cudaStream_t s);
void field_unpack(const cd* y, const double* inv_eta, int64_t n, int64_t m, int nrhs, bool c64, void* u,
                  cudaStream_t s);

QuadRule make_quad_rule(const MediumDev& m);

// stage timers (api.cu): begin/end record events on the stream when profiling is on;
// flush synchronises the stream and accumulates the elapsed times.
void prof_begin(lfmm_geometry_s* g, Stage st, cudaStream_t s);
void prof_end(lfmm_geometry_s* g, Stage st, cudaStream_t s);
void prof_flush(lfmm_geometry_s* g, cudaStream_t s);

}  // namespace lfmm
