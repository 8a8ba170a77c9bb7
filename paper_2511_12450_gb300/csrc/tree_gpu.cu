// tree_gpu.cu -- the quadtree and every interaction list built on the GPU.
//
// It implements the tree definition of tree.cpp (Sec. 4.1 leaves its parameters open;
// tree.cpp states the reading) and gives the same integers bit for bit: the root
// square, the quantised coordinates, the depth, the point order, the boxes of every
// level and the free-space and reaction lists in the same order.  Every floating-point
// decision (quantisation, cell bounds, reaction-centre heights, the far test) is taken
// with explicitly rounded operations (__dadd_rn, __dmul_rn, ...) in the host's order,
// so no contraction into a fused multiply-add can move a boundary case.
//
// Steps (all on the calling thread's per-thread stream):
//  1. bounding box by min/max reduction; W, x0, y0 on the host from the four values;
//  2. 20-bit quantisation; keys (layer, Morton code at level 18), sorted; for each level
//     the longest run of equal (layer, cell) keys by binary search -> the depth D;
//  3. point order: stable LSD radix sort (8-bit digits) of (layer, Morton at level D)
//     over the input order, so equal keys keep the input order;
//  4. boxes level by level: a box starts where the (layer, cell) of consecutive sorted
//     points changes; scans number them; parents and child ranges follow;
//  5. lists level by level with a count pass, a scan and a fill pass: candidates are the
//     children of the parent's near list, in the order of that list.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <stdexcept>
#include <vector>

#include "geometry.h"

namespace lfmm {

static const int GT_QBITS = 20;
static const int GT_DCAP = 18;
static const int GT_PCAP = 80;
static const int GT_L0MIN = 2;

// ---------------------------------------------------------------------------- device buffers
template <class T>
struct DevVec {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t s = cudaStreamPerThread;
    DevVec() = default;
    explicit DevVec(size_t count) { resize(count); }
    void resize(size_t count) {
        release();
        n = count;
        cuda_check(cudaMallocAsync((void**)&p, sizeof(T) * std::max<size_t>(count, 1), s), "cudaMallocAsync (tree)");
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
    }
    ~DevVec() { release(); }
    DevVec(const DevVec&) = delete;
    DevVec& operator=(const DevVec&) = delete;
    std::vector<T> host(size_t count) const {
        std::vector<T> h(count);
        if (count) cuda_check(cudaMemcpyAsync(h.data(), p, sizeof(T) * count, cudaMemcpyDeviceToHost, s), "tree d2h");
        cuda_check(cudaStreamSynchronize(s), "tree d2h");
        return h;
    }
};

static inline int grid_for(int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 32));
}

// ---------------------------------------------------------------------------- scan
// exclusive scan of int counts (64-bit offsets), in three passes over blocks of SCAN_B
#define SCAN_B 1024
__global__ void k_scan_blocks(const int* __restrict__ in, int64_t n, int64_t* __restrict__ out,
                              int64_t* __restrict__ block_sum) {
    __shared__ int64_t sh[SCAN_B];
    const int64_t base = (int64_t)blockIdx.x * SCAN_B;
    for (int i = threadIdx.x; i < SCAN_B; i += blockDim.x) sh[i] = (base + i < n) ? in[base + i] : 0;
    __syncthreads();
    if (threadIdx.x == 0) {   // serial over the block: exact and ordered (set-up only)
        int64_t acc = 0;
        for (int i = 0; i < SCAN_B; ++i) { const int64_t v = sh[i]; sh[i] = acc; acc += v; }
        block_sum[blockIdx.x] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_B; i += blockDim.x)
        if (base + i < n) out[base + i] = sh[i];
}
__global__ void k_scan_sums(int64_t* __restrict__ block_sum, int64_t nb, int64_t* __restrict__ total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t acc = 0;
    for (int64_t b = 0; b < nb; ++b) { const int64_t v = block_sum[b]; block_sum[b] = acc; acc += v; }
    *total = acc;
}
__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ block_sum) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] += block_sum[i / SCAN_B];
}
// out[0..n) = exclusive prefix sums of in, out[n] = total; returns the total
static int64_t exclusive_scan(const int* in, int64_t n, DevVec<int64_t>& out) {
    cudaStream_t s = cudaStreamPerThread;
    out.resize(n + 1);
    const int64_t nb = (n + SCAN_B - 1) / SCAN_B;
    DevVec<int64_t> bs(nb + 1);
    if (n > 0) {
        k_scan_blocks<<<(int)nb, 256, 0, s>>>(in, n, out.p, bs.p);
        k_scan_sums<<<1, 32, 0, s>>>(bs.p, nb, out.p + n);
        k_scan_add<<<grid_for(n), 256, 0, s>>>(out.p, n, bs.p);
        cuda_check(cudaGetLastError(), "tree scan");
    } else {
        cuda_check(cudaMemsetAsync(out.p, 0, sizeof(int64_t), s), "tree scan");
    }
    int64_t total = 0;
    cuda_check(cudaMemcpyAsync(&total, out.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "scan total");
    cuda_check(cudaStreamSynchronize(s), "scan total");
    return total;
}

// ---------------------------------------------------------------------------- radix sort
// Stable LSD radix sort of 64-bit keys (the low `bits` bits) with int values, 8-bit
// digits.  A tile of RS_TILE consecutive items belongs to one warp, which ranks its items
// in rounds of 32 in their order (__match_any_sync), so equal digits keep their order.
#define RS_TILE 1024
__global__ void __launch_bounds__(32) k_rs_hist(const uint64_t* __restrict__ key, int64_t n, int shift,
                                                int* __restrict__ hist, int ntile) {
    __shared__ int h[256];
    for (int d = threadIdx.x; d < 256; d += 32) h[d] = 0;
    __syncwarp();
    const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    for (int r = threadIdx.x; r < RS_TILE; r += 32) {
        const int64_t i = t0 + r;
        if (i < n) atomicAdd(&h[(int)((key[i] >> shift) & 255u)], 1);
    }
    __syncwarp();
    for (int d = threadIdx.x; d < 256; d += 32) hist[(int64_t)d * ntile + blockIdx.x] = h[d];
}
__global__ void __launch_bounds__(32) k_rs_scatter(const uint64_t* __restrict__ key, const int* __restrict__ val,
                                                   int64_t n, int shift, const int64_t* __restrict__ off, int ntile,
                                                   uint64_t* __restrict__ key_out, int* __restrict__ val_out) {
    __shared__ int64_t base[256];
    const int lane = threadIdx.x;
    for (int d = lane; d < 256; d += 32) base[d] = off[(int64_t)d * ntile + blockIdx.x];
    __syncwarp();
    const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    for (int r0 = 0; r0 < RS_TILE; r0 += 32) {
        const int64_t i = t0 + r0 + lane;
        const bool valid = i < n;
        const unsigned mask = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const uint64_t k = key[i];
            const int d = (int)((k >> shift) & 255u);
            const unsigned peers = __match_any_sync(mask, d);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            const int64_t pos = base[d] + rank;
            key_out[pos] = k;
            if (val) val_out[pos] = val[i];
            __syncwarp(mask);
            if (rank == 0) base[d] += __popc(peers);
        }
        __syncwarp();
    }
}
// sorts (key, val) in place (val may be null), considering the low `bits` bits
static void radix_sort(DevVec<uint64_t>& key, DevVec<int>* val, int64_t n, int bits) {
    cudaStream_t s = cudaStreamPerThread;
    if (n <= 1) return;
    const int ntile = (int)((n + RS_TILE - 1) / RS_TILE);
    DevVec<uint64_t> k2(n);
    DevVec<int> v2(val ? n : 1);
    DevVec<int> hist((size_t)256 * ntile);
    DevVec<int64_t> off;
    uint64_t *ka = key.p, *kb = k2.p;
    int *va = val ? val->p : nullptr, *vb = val ? v2.p : nullptr;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<ntile, 32, 0, s>>>(ka, n, shift, hist.p, ntile);
        cuda_check(cudaGetLastError(), "k_rs_hist");
        exclusive_scan(hist.p, (int64_t)256 * ntile, off);
        k_rs_scatter<<<ntile, 32, 0, s>>>(ka, va, n, shift, off.p, ntile, kb, vb);
        cuda_check(cudaGetLastError(), "k_rs_scatter");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != key.p) {
        cuda_check(cudaMemcpyAsync(key.p, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s), "sort copy");
        if (val) cuda_check(cudaMemcpyAsync(val->p, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, s), "sort copy");
    }
}

// ---------------------------------------------------------------------------- points
__device__ __forceinline__ uint64_t spread_bits(uint32_t v) {
    uint64_t x = v;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}
// x bit b -> key bit 2b, y bit b -> key bit 2b + 1 (as tree.cpp's morton2)
__device__ __forceinline__ uint64_t morton_dev(uint32_t ix, uint32_t iy) { return spread_bits(ix) | (spread_bits(iy) << 1); }

__global__ void k_minmax(const double* __restrict__ px, const double* __restrict__ py, int64_t n,
                         double* __restrict__ part) {
    __shared__ double sh[4][256];
    double a = px[0], b = px[0], c = py[0], d = py[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        a = fmin(a, px[i]); b = fmax(b, px[i]); c = fmin(c, py[i]); d = fmax(d, py[i]);
    }
    sh[0][threadIdx.x] = a; sh[1][threadIdx.x] = b; sh[2][threadIdx.x] = c; sh[3][threadIdx.x] = d;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] = fmin(sh[0][threadIdx.x], sh[0][threadIdx.x + o]);
            sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + o]);
            sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + o]);
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 4; ++q) part[4 * blockIdx.x + q] = sh[q][0];
}
// q = floor(((x - x0) / W) * 2^20), clamped: the host's expression, each operation rounded
__global__ void k_quantize(const double* __restrict__ px, const double* __restrict__ py, int64_t n, double x0,
                           double y0, double W, uint32_t* __restrict__ qx, uint32_t* __restrict__ qy) {
    const double scale = (double)(1u << GT_QBITS);
    const int64_t qmax = (1 << GT_QBITS) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double fx = floor(__dmul_rn(__ddiv_rn(__dsub_rn(px[i], x0), W), scale));
        const double fy = floor(__dmul_rn(__ddiv_rn(__dsub_rn(py[i], y0), W), scale));
        const int64_t a = (int64_t)fx, b = (int64_t)fy;
        qx[i] = (uint32_t)min(max(a, (int64_t)0), qmax);
        qy[i] = (uint32_t)min(max(b, (int64_t)0), qmax);
    }
}
// key = layer << 2 lev | Morton code of the level-lev cell
__global__ void k_cell_keys(const uint32_t* __restrict__ qx, const uint32_t* __restrict__ qy,
                            const int* __restrict__ layer, int64_t n, int lev, uint64_t* __restrict__ key,
                            int* __restrict__ idx) {
    const int sh = GT_QBITS - lev;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = ((uint64_t)layer[i] << (2 * lev)) | morton_dev(qx[i] >> sh, qy[i] >> sh);
        if (idx) idx[i] = (int)i;
    }
}
// longest run of equal (layer, level-l cell) among the keys sorted at level 18
__global__ void k_max_run(const uint64_t* __restrict__ key, int64_t n, int l, int* __restrict__ maxrun) {
    const int shift = 2 * (GT_DCAP - l);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key[i] >> shift;
        if (i > 0 && (key[i - 1] >> shift) == k) continue;   // not the first point of its cell
        int64_t lo = i, hi = n;                                // first index whose cell is past k
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((key[mid] >> shift) <= k) lo = mid + 1;
            else hi = mid;
        }
        const int64_t run = lo - i;
        atomicMax(maxrun, run > 0x7fffffff ? 0x7fffffff : (int)run);
    }
}

// ---------------------------------------------------------------------------- boxes
// flag[s] = 1 where the (layer, level-l cell) of sorted point s differs from s - 1
__global__ void k_box_flags(const uint64_t* __restrict__ keyD, int64_t n, int shift, int* __restrict__ flag) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        flag[s] = (s == 0 || (keyD[s] >> shift) != (keyD[s - 1] >> shift)) ? 1 : 0;
}
// boxes of level l: begin, layer, cell, parent; the level's box index of every point
__global__ void k_box_make(const int* __restrict__ flag, const int64_t* __restrict__ ex, int64_t n, int l, int base,
                           int base_prev, const int* __restrict__ perm, const int* __restrict__ layer,
                           const uint32_t* __restrict__ qx, const uint32_t* __restrict__ qy,
                           const int* __restrict__ pt_box_prev, int* __restrict__ pt_box, int* __restrict__ b_level,
                           int* __restrict__ b_layer, int* __restrict__ b_ix, int* __restrict__ b_iy,
                           int* __restrict__ b_begin, int* __restrict__ b_parent) {
    const int sh = GT_QBITS - l;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int bi = (int)(ex[s] + flag[s] - 1);   // index of s's box within the level
        pt_box[s] = bi;
        if (!flag[s]) continue;
        const int b = base + bi, i = perm[s];
        b_level[b] = l;
        b_layer[b] = layer[i];
        b_ix[b] = (int)(qx[i] >> sh);
        b_iy[b] = (int)(qy[i] >> sh);
        b_begin[b] = (int)s;
        b_parent[b] = (l > 0) ? base_prev + pt_box_prev[s] : -1;
    }
}
__global__ void k_box_end(const int* __restrict__ b_begin, int b0, int b1, int n, int* __restrict__ b_end) {
    for (int b = b0 + blockIdx.x * blockDim.x + threadIdx.x; b < b1; b += gridDim.x * blockDim.x)
        b_end[b] = (b + 1 < b1) ? b_begin[b + 1] : n;
}
__global__ void k_children(const int* __restrict__ b_parent, int b0, int b1, int* __restrict__ c_begin,
                           int* __restrict__ c_end) {
    for (int b = b0 + blockIdx.x * blockDim.x + threadIdx.x; b < b1; b += gridDim.x * blockDim.x) {
        const int p = b_parent[b];
        if (b == b0 || b_parent[b - 1] != p) c_begin[p] = b;
        if (b + 1 == b1 || b_parent[b + 1] != p) c_end[p] = b + 1;
    }
}

// ---------------------------------------------------------------------------- lists
// Reaction-centre heights and the far test, with the host's operations in its order.
__device__ __forceinline__ double clipped_height_dev(double yif, bool above, double lo, double hi) {
    if (above) return __dsub_rn(__dmul_rn(0.5, __dadd_rn(fmax(lo, yif), hi)), yif);
    return __dsub_rn(yif, __dmul_rn(0.5, __dadd_rn(lo, fmin(hi, yif))));
}
struct CompDev {
    int ls, a, lt, b;
    double Hc, ky_tab;
};
struct ListCtx {
    // boxes
    const int *b_layer, *b_ix, *b_iy, *b_parent, *c_begin, *c_end;
    double y0, w;       // root corner and the level's cell width
    int l, l0, base, nbl, ncomp, base_prev;
    MediumDev med;
    const CompDev* comps;
    // the previous level's near lists: CSR over its items (box, component)
    const int64_t* prev_ptr;
    const int* prev_idx;
    int level0_of_layer[LFMM_MAXLAY];   // level-0 box of each layer (-1 if none)
};
__device__ __forceinline__ bool react_far(const ListCtx& c, const CompDev& C, int S, int T) {
    const double loS = __dadd_rn(c.y0, __dmul_rn((double)c.b_iy[S], c.w));
    const double hiS = __dadd_rn(c.y0, __dmul_rn((double)(c.b_iy[S] + 1), c.w));
    const double loT = __dadd_rn(c.y0, __dmul_rn((double)c.b_iy[T], c.w));
    const double hiT = __dadd_rn(c.y0, __dmul_rn((double)(c.b_iy[T] + 1), c.w));
    const double hS = (C.a == 0) ? clipped_height_dev(c.med.yint[C.ls], true, loS, hiS)
                                 : clipped_height_dev(c.med.yint[C.ls - 1], false, loS, hiS);
    const double hT = (C.b == 0) ? clipped_height_dev(c.med.yint[C.lt - 1], false, loT, hiT)
                                 : clipped_height_dev(c.med.yint[C.lt], true, loT, hiT);
    const double Dc = __dadd_rn(__dadd_rn(hS, hT), C.Hc);
    const bool col = abs(c.b_ix[S] - c.b_ix[T]) >= 2 && __dmul_rn(C.ky_tab, __dsub_rn(c.w, Dc)) <= REACT_COND_EXP;
    return col || Dc >= __dmul_rn(__dmul_rn(2.0, c.w), 1.0 - 1e-9);
}
// One item = (box T of the level, component c); c = -1 / ncomp = 0 means the free-space
// lists (same layer, near = touching cells).  Pass 0 counts, pass 1 writes, in the host's
// candidate order: the children of each box of the parent's near list, in list order.
template <bool REACT>
__global__ void k_lists(ListCtx c, int pass, int* __restrict__ ncnt, int* __restrict__ vcnt,
                        const int64_t* __restrict__ nptr, int* __restrict__ nidx, const int64_t* __restrict__ vptr,
                        int* __restrict__ vidx, int* __restrict__ vcomp) {
    const int nc = REACT ? c.ncomp : 1;
    const int64_t nitem = (int64_t)c.nbl * nc;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < nitem; it += (int64_t)gridDim.x * blockDim.x) {
        const int ti = (int)(it / nc), ci = (int)(it - (int64_t)ti * nc);
        const int T = c.base + ti;
        int nn = 0, nv = 0;
        int64_t no = 0, vo = 0;
        if (pass == 1) { no = nptr[it]; vo = vptr[it]; }
        CompDev C{};
        bool active = true;
        if (REACT) {
            C = c.comps[ci];
            active = c.b_layer[T] == C.lt;
        }
        if (active) {
            auto visit = [&](int S) {
                bool near;
                if (c.l < c.l0) near = true;
                else if (REACT) near = !react_far(c, C, S, T);
                else near = abs(c.b_ix[S] - c.b_ix[T]) <= 1 && abs(c.b_iy[S] - c.b_iy[T]) <= 1;
                if (near) {
                    if (pass == 1) nidx[no + nn] = S;
                    ++nn;
                } else {
                    if (pass == 1) { vidx[vo + nv] = S; if (REACT) vcomp[vo + nv] = ci; }
                    ++nv;
                }
            };
            if (c.l == 0) {
                if (REACT) {
                    const int S = c.level0_of_layer[C.ls];
                    if (S >= 0) visit(S);
                } else {
                    visit(T);
                }
            } else {
                const int64_t pi = (int64_t)(c.b_parent[T] - c.base_prev) * nc + ci;
                for (int64_t k = c.prev_ptr[pi]; k < c.prev_ptr[pi + 1]; ++k) {
                    const int S = c.prev_idx[k];
                    for (int ch = c.c_begin[S]; ch < c.c_end[S]; ++ch) visit(ch);
                }
            }
        }
        if (pass == 0) { ncnt[it] = nn; vcnt[it] = nv; }
    }
}

// ---------------------------------------------------------------------------- driver
void build_tree_gpu(TreeHost& t, const double* d_px, const double* d_py, const int* d_layer, int64_t n,
                    const MediumDev& med, int p, int leaf_size) {
    cudaStream_t s = cudaStreamPerThread;
    if (n <= 0) throw std::runtime_error("build_tree: no points");
    // 1. root square
    {
        const int nb = std::min<int64_t>((n + 255) / 256, 1024);
        DevVec<double> part((size_t)4 * nb);
        k_minmax<<<nb, 256, 0, s>>>(d_px, d_py, n, part.p);
        cuda_check(cudaGetLastError(), "k_minmax");
        std::vector<double> h = part.host((size_t)4 * nb);
        double xmin = h[0], xmax = h[1], ymin = h[2], ymax = h[3];
        for (int b = 1; b < nb; ++b) {
            xmin = std::min(xmin, h[4 * b]); xmax = std::max(xmax, h[4 * b + 1]);
            ymin = std::min(ymin, h[4 * b + 2]); ymax = std::max(ymax, h[4 * b + 3]);
        }
        const double ext = std::max(xmax - xmin, ymax - ymin);
        const double W = ext > 0 ? ext * (1.0 + 1.0 / 1024.0) : 1.0;
        const double cx = 0.5 * (xmin + xmax), cy = 0.5 * (ymin + ymax);
        t.W = W;
        t.x0 = cx - 0.5 * W;
        t.y0 = cy - 0.5 * W;
    }
    DevVec<uint32_t> qx(n), qy(n);
    k_quantize<<<grid_for(n), 256, 0, s>>>(d_px, d_py, n, t.x0, t.y0, t.W, qx.p, qy.p);
    cuda_check(cudaGetLastError(), "k_quantize");
    // 2. depth: the smallest level with at most leaf_size points per (layer, cell)
    int D = GT_DCAP;
    {
        DevVec<uint64_t> key(n);
        k_cell_keys<<<grid_for(n), 256, 0, s>>>(qx.p, qy.p, d_layer, n, GT_DCAP, key.p, nullptr);
        cuda_check(cudaGetLastError(), "k_cell_keys");
        radix_sort(key, nullptr, n, 4 + 2 * GT_DCAP);
        DevVec<int> runs(GT_DCAP + 1);
        cuda_check(cudaMemsetAsync(runs.p, 0, sizeof(int) * (GT_DCAP + 1), s), "memset runs");
        for (int l = 0; l <= GT_DCAP; ++l) k_max_run<<<grid_for(n), 256, 0, s>>>(key.p, n, l, runs.p + l);
        cuda_check(cudaGetLastError(), "k_max_run");
        const std::vector<int> worst = runs.host(GT_DCAP + 1);
        for (int l = 0; l <= GT_DCAP; ++l)
            if (worst[l] <= leaf_size) { D = l; break; }
    }
    t.D = D;
    t.p_level.assign(D + 1, p);
    for (int l = 0; l <= D; ++l) {
        double kr = med.kmax * (t.W / (double)(1u << l)) * 0.70710678118654752;
        int pl = (int)std::ceil(kr + 9.0 * std::pow(kr, 1.0 / 3.0));
        t.p_level[l] = std::max(p, pl);
    }
    t.l0 = D + 1;
    for (int l = GT_L0MIN; l <= D; ++l)
        if (t.p_level[l] <= GT_PCAP) { t.l0 = l; break; }
    // 3. point order: (layer, Morton at level D, input index)
    DevVec<uint64_t> keyD(n);
    DevVec<int> perm(n);
    k_cell_keys<<<grid_for(n), 256, 0, s>>>(qx.p, qy.p, d_layer, n, D, keyD.p, perm.p);
    cuda_check(cudaGetLastError(), "k_cell_keys");
    radix_sort(keyD, &perm, n, 4 + 2 * D);
    t.perm = perm.host(n);
    {
        std::vector<int> lay_in(n);
        cuda_check(cudaMemcpyAsync(lay_in.data(), d_layer, sizeof(int) * n, cudaMemcpyDeviceToHost, s), "layers");
        cuda_check(cudaStreamSynchronize(s), "layers");
        t.layer_sorted.resize(n);
        for (int64_t q = 0; q < n; ++q) t.layer_sorted[q] = lay_in[t.perm[q]];
    }
    // 4. boxes: count per level, then make them
    DevVec<int> flag(n);
    std::vector<DevVec<int64_t>> ex(D + 1);
    t.level_start.assign(D + 2, 0);
    for (int l = 0; l <= D; ++l) {
        k_box_flags<<<grid_for(n), 256, 0, s>>>(keyD.p, n, 2 * (D - l), flag.p);
        cuda_check(cudaGetLastError(), "k_box_flags");
        // flags are recomputed below; only the counts are kept here
        const int64_t cnt = exclusive_scan(flag.p, n, ex[l]);
        t.level_start[l + 1] = t.level_start[l] + (int)cnt;
    }
    const int nb = t.level_start[D + 1];
    t.nbox = nb;
    DevVec<int> b_level(nb), b_layer(nb), b_ix(nb), b_iy(nb), b_begin(nb), b_end(nb), b_parent(nb), c_begin(nb),
        c_end(nb);
    cuda_check(cudaMemsetAsync(c_begin.p, 0, sizeof(int) * nb, s), "memset");
    cuda_check(cudaMemsetAsync(c_end.p, 0, sizeof(int) * nb, s), "memset");
    DevVec<int> ptbox_a(n), ptbox_b(n);
    int* pt_prev = ptbox_a.p;
    int* pt_cur = ptbox_b.p;
    for (int l = 0; l <= D; ++l) {
        k_box_flags<<<grid_for(n), 256, 0, s>>>(keyD.p, n, 2 * (D - l), flag.p);
        k_box_make<<<grid_for(n), 256, 0, s>>>(flag.p, ex[l].p, n, l, t.level_start[l],
                                               l > 0 ? t.level_start[l - 1] : 0, perm.p, d_layer, qx.p, qy.p,
                                               pt_prev, pt_cur, b_level.p, b_layer.p, b_ix.p, b_iy.p, b_begin.p,
                                               b_parent.p);
        const int b0 = t.level_start[l], b1 = t.level_start[l + 1];
        k_box_end<<<grid_for(b1 - b0), 256, 0, s>>>(b_begin.p, b0, b1, (int)n, b_end.p);
        if (l > 0) k_children<<<grid_for(b1 - b0), 256, 0, s>>>(b_parent.p, b0, b1, c_begin.p, c_end.p);
        cuda_check(cudaGetLastError(), "tree boxes");
        std::swap(pt_prev, pt_cur);
    }
    t.box_level = b_level.host(nb);
    t.box_layer = b_layer.host(nb);
    t.box_ix = b_ix.host(nb);
    t.box_iy = b_iy.host(nb);
    t.box_begin = b_begin.host(nb);
    t.box_end = b_end.host(nb);
    t.box_parent = b_parent.host(nb);
    t.child_begin = c_begin.host(nb);
    t.child_end = c_end.host(nb);
    // reaction components (the same enumeration as tree.cpp)
    t.comps.clear();
    const int L = med.nl - 1;
    for (int ls = 0; ls <= L; ++ls)
        for (int a = 0; a < 2; ++a) {
            if (a == 0 && ls >= L) continue;
            if (a == 1 && ls <= 0) continue;
            for (int lt = 0; lt <= L; ++lt)
                for (int b = 0; b < 2; ++b) {
                    if (b == 0 && lt <= 0) continue;
                    if (b == 1 && lt >= L) continue;
                    t.comps.push_back(Component{ls, a, lt, b, comp_extra_thickness(med, ls, a, lt, b)});
                }
        }
    const int ncomp = (int)t.comps.size();
    std::vector<CompDev> hc(std::max(ncomp, 1));
    const double t_tab = table_detour_end(med);
    for (int c = 0; c < ncomp; ++c) {
        const Component& C = t.comps[c];
        const double kl = std::min(med.k[C.ls], med.k[C.lt]);
        hc[c] = CompDev{C.ls, C.a, C.lt, C.b, C.Hc, std::sqrt(t_tab * t_tab - kl * kl)};
    }
    DevVec<CompDev> d_comps(hc.size());
    cuda_check(cudaMemcpyAsync(d_comps.p, hc.data(), sizeof(CompDev) * hc.size(), cudaMemcpyHostToDevice, s), "comps");
    // 5. lists, level by level (free space: one item per box; reaction: per (box, component))
    ListCtx base{};
    base.b_layer = b_layer.p; base.b_ix = b_ix.p; base.b_iy = b_iy.p; base.b_parent = b_parent.p;
    base.c_begin = c_begin.p; base.c_end = c_end.p;
    base.y0 = t.y0;
    base.l0 = t.l0;
    base.med = med;
    base.comps = d_comps.p;
    for (int q = 0; q < LFMM_MAXLAY; ++q) base.level0_of_layer[q] = -1;
    for (int b = t.level_start[0]; b < t.level_start[1]; ++b) base.level0_of_layer[t.box_layer[b]] = b;
    for (int react = 0; react < 2; ++react) {
        const int nc = react ? ncomp : 1;
        if (react && ncomp == 0) {
            t.vreact_ptr.assign(nb + 1, 0);
            t.ureact_ptr.assign(nb + 1, 0);
            t.vreact_idx.clear(); t.vreact_comp.clear(); t.ureact_idx.clear(); t.ureact_comp.clear();
            break;
        }
        std::vector<int> vptr_all(1, 0), vidx_all, vcomp_all;
        std::vector<int64_t> near_item_ptr_D;
        std::vector<int> near_idx_D;
        DevVec<int64_t> prev_ptr(1);
        DevVec<int> prev_idx(1);
        cuda_check(cudaMemsetAsync(prev_ptr.p, 0, sizeof(int64_t), s), "memset");
        for (int l = 0; l <= D; ++l) {
            ListCtx c = base;
            c.l = l;
            c.w = t.W / (double)(1u << l);
            c.base = t.level_start[l];
            c.nbl = t.level_start[l + 1] - t.level_start[l];
            c.ncomp = ncomp;
            c.base_prev = l > 0 ? t.level_start[l - 1] : 0;
            c.prev_ptr = prev_ptr.p;
            c.prev_idx = prev_idx.p;
            const int64_t nitem = (int64_t)c.nbl * nc;
            DevVec<int> ncnt(nitem), vcnt(nitem);
            if (react) k_lists<true><<<grid_for(nitem), 256, 0, s>>>(c, 0, ncnt.p, vcnt.p, nullptr, nullptr, nullptr, nullptr, nullptr);
            else k_lists<false><<<grid_for(nitem), 256, 0, s>>>(c, 0, ncnt.p, vcnt.p, nullptr, nullptr, nullptr, nullptr, nullptr);
            cuda_check(cudaGetLastError(), "k_lists count");
            DevVec<int64_t> nptr, vptr;
            const int64_t ntot = exclusive_scan(ncnt.p, nitem, nptr);
            const int64_t vtot = exclusive_scan(vcnt.p, nitem, vptr);
            DevVec<int> nidx(ntot), vidx(vtot), vcomp(react ? vtot : 1);
            if (react) k_lists<true><<<grid_for(nitem), 256, 0, s>>>(c, 1, nullptr, nullptr, nptr.p, nidx.p, vptr.p, vidx.p, vcomp.p);
            else k_lists<false><<<grid_for(nitem), 256, 0, s>>>(c, 1, nullptr, nullptr, nptr.p, nidx.p, vptr.p, vidx.p, nullptr);
            cuda_check(cudaGetLastError(), "k_lists fill");
            // the level's far lists: per box, its items' entries one after another
            const std::vector<int64_t> hv = vptr.host(nitem + 1);
            const std::vector<int> hvi = vidx.host(vtot);
            std::vector<int> hvc;
            if (react) hvc = vcomp.host(vtot);
            for (int ti = 0; ti < c.nbl; ++ti) vptr_all.push_back((int)hv[(int64_t)(ti + 1) * nc]);
            const int add = (int)vidx_all.size();
            for (int q = (int)vptr_all.size() - c.nbl; q < (int)vptr_all.size(); ++q) vptr_all[q] += add;
            vidx_all.insert(vidx_all.end(), hvi.begin(), hvi.end());
            if (react) vcomp_all.insert(vcomp_all.end(), hvc.begin(), hvc.end());
            if (l == D) {
                near_item_ptr_D = nptr.host(nitem + 1);
                near_idx_D = nidx.host(ntot);
            }
            prev_ptr.resize(nitem + 1);
            cuda_check(cudaMemcpyAsync(prev_ptr.p, nptr.p, sizeof(int64_t) * (nitem + 1), cudaMemcpyDeviceToDevice, s),
                       "near ptr");
            prev_idx.resize(std::max<int64_t>(ntot, 1));
            if (ntot)
                cuda_check(cudaMemcpyAsync(prev_idx.p, nidx.p, sizeof(int) * ntot, cudaMemcpyDeviceToDevice, s),
                           "near idx");
        }
        // near lists of the leaves (level D), as CSR over all boxes
        std::vector<int> uptr(nb + 1, 0), uidx, ucomp;
        const int leaf0 = t.level_start[D];
        for (int b = 0; b < nb; ++b) {
            if (b >= leaf0) {
                const int ti = b - leaf0;
                for (int ci = 0; ci < nc; ++ci) {
                    const int64_t it = (int64_t)ti * nc + ci;
                    for (int64_t k = near_item_ptr_D[it]; k < near_item_ptr_D[it + 1]; ++k) {
                        uidx.push_back(near_idx_D[k]);
                        if (react) ucomp.push_back(ci);
                    }
                }
            }
            uptr[b + 1] = (int)uidx.size();
        }
        if (react) {
            t.vreact_ptr = vptr_all; t.vreact_idx = vidx_all; t.vreact_comp = vcomp_all;
            t.ureact_ptr = uptr; t.ureact_idx = uidx; t.ureact_comp = ucomp;
        } else {
            t.vfree_ptr = vptr_all; t.vfree_idx = vidx_all;
            t.ufree_ptr = uptr; t.ufree_idx = uidx;
        }
    }
    cuda_check(cudaStreamSynchronize(s), "tree");
}

}  // namespace lfmm
