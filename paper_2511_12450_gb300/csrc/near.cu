// near.cu -- near-field part of the Nystrom operator (Sec. 3.3, eqs. matrixelmemts,
// Llayerscomponent; Sec. 4.1 near-field interactions).
//
// For every target leaf T the near field is a row of dense blocks, one per
// source leaf S that is near T for the free-space part (same layer, touching
// cells) or for at least one reaction component (image-frame neighbours).
// Block (T, S) holds, for target point i in T and source point j in S,
//   |Gamma_j| (i/4) H_0(k |c_i - c_j|)                 free space, same layer, j != i
//   I^s_i                                               j == i (analytic self term)
//   |Gamma_j| sum_c K_c(x_j - x_i, h_s(y_j), h_t(y_i))  reaction components near in the image frame
// and acts on Phi directly.  In the combined-field form (opt-in) every entry is
// |Gamma_j| [n_j . grad_{c_j} - i k] of the same kernels, and the diagonal is
// 1/2 - i k I^s (devmath.cuh: free_kernel, self_entry; sommerfeld.cuh:
// react_kernel_grad_warp).  The blocks are computed once at set-up (Sommerfeld
// quadrature for the reaction entries) and stored column-major, so the per
// matvec near field is one streaming block-sparse product bounded by HBM
// bandwidth.
#include <cuda_runtime.h>

#include <algorithm>
#include <stdexcept>
#include <vector>

#include "geometry.h"
#include "sommerfeld.cuh"

namespace lfmm {

struct NearTask {   // the reaction entries of one block
    int blk;        // block index
    int c0, c1;     // its components: [c0, c1) of the component list
    int64_t first;  // first entry index in the flattened task space
};

// free-space entries and the self term; initialises every block
__global__ void k_near_free(MediumDev m, const int* __restrict__ blk_tgt, const int* __restrict__ blk_src,
                            const int64_t* __restrict__ blk_off, const unsigned char* __restrict__ blk_free,
                            const int* __restrict__ box_begin, const int* __restrict__ box_end,
                            const int* __restrict__ box_layer, const double* __restrict__ px,
                            const double* __restrict__ py, const double* __restrict__ pw,
                            const double* __restrict__ nx, const double* __restrict__ ny, cd* __restrict__ val) {
    const bool cf = nx != nullptr;
    const int blk = blockIdx.x;
    const int T = blk_tgt[blk], S = blk_src[blk];
    const int tb = box_begin[T], nT = box_end[T] - tb;
    const int sb = box_begin[S], nS = box_end[S] - sb;
    const bool fr = blk_free[blk] != 0;
    const double k = m.k[box_layer[T]];
    cd* v = val + blk_off[blk];
    for (int e = threadIdx.x; e < nT * nS; e += blockDim.x) {
        int i = e % nT, j = e / nT;
        cd out = mk(0.0, 0.0);
        if (fr) {
            int pi = tb + i, pj = sb + j;
            if (pw[pj] == 0.0) {
                // a field point (weight 0) is never a source; its own diagonal is 0
            } else if (pi == pj) {
                out = self_entry(k, pw[pi], cf);
            } else {
                out = pw[pj] * free_kernel(k, px[pj] - px[pi], py[pj] - py[pi], cf, cf ? nx[pj] : 0.0,
                                           cf ? ny[pj] : 0.0);
            }
        }
        v[(int64_t)j * nT + i] = out;
    }
}

// reaction entries: one warp per (block, entry); the warp adds the entry's components in
// their list order and writes once, so the stored values do not depend on scheduling
__global__ void k_near_react(MediumDev m, QuadRule q, const NearTask* __restrict__ tasks, int ntask,
                             int64_t nwork, const int* __restrict__ task_comp, const int* __restrict__ blk_tgt,
                             const int* __restrict__ blk_src, const int64_t* __restrict__ blk_off,
                             const int* __restrict__ comp, const double* __restrict__ comp_H,
                             const int* __restrict__ box_begin, const int* __restrict__ box_end,
                             const double* __restrict__ px, const double* __restrict__ py,
                             const double* __restrict__ pw, const double* __restrict__ nx,
                             const double* __restrict__ ny, cd* __restrict__ val) {
    const bool cf = nx != nullptr;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wk = warp; wk < nwork; wk += nwarps) {
        // locate the block by binary search on first
        int lo = 0, hi = ntask - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (tasks[mid].first <= wk) lo = mid; else hi = mid - 1;
        }
        const NearTask tk = tasks[lo];
        const int T = blk_tgt[tk.blk], S = blk_src[tk.blk];
        const int tb = box_begin[T], nT = box_end[T] - tb;
        const int sb = box_begin[S];
        const int64_t e = wk - tk.first;
        const int i = (int)(e % nT), j = (int)(e / nT);
        const int pi = tb + i, pj = sb + j;
        if (pw[pj] == 0.0) continue;   // a field point (weight 0) is never a source (uniform per warp)
        const double X = px[pj] - px[pi];
        cd Ksum = mk(0.0, 0.0);
        for (int q2 = tk.c0; q2 < tk.c1; ++q2) {
            const int c = task_comp[q2];
            const int ls = comp[4 * c], a = comp[4 * c + 1], lt = comp[4 * c + 2], b = comp[4 * c + 3];
            const double hs = (a == 0) ? (py[pj] - m.yint[ls]) : (m.yint[ls - 1] - py[pj]);
            const double ht = (b == 0) ? (m.yint[lt - 1] - py[pi]) : (py[pi] - m.yint[lt]);
            if (cf) {
                cd gk[3];
                react_kernel_grad_warp(m, q, ls, a, lt, b, comp_H[c], X, hs, ht, gk);
                Ksum += react_cf_combine(gk, a, m.k[ls], nx[pj], ny[pj]);
            } else {
                Ksum += react_kernel_warp(m, q, ls, a, lt, b, comp_H[c], X, hs, ht);
            }
        }
        if ((threadIdx.x & 31) == 0) {
            cd* dst = val + blk_off[tk.blk] + (int64_t)j * nT + i;
            *dst += pw[pj] * Ksum;
        }
    }
}

// y_T += (near row of leaf T) x, one CTA of NW warps per target leaf.
//
// The blocks of one target leaf T are stored one after another, each column-major
// with leading dimension nT = |T|, so together they form one column-major nT x nJ
// matrix whose column c multiplies x at the sorted position J[c].  Warp w takes the
// contiguous share [c0 + nJ w / NW, c0 + nJ (w + 1) / NW) of the columns, and the rows
// in chunks of r = min(32, nT): G = 32 / r groups of r lanes each walk every G-th
// column of its share (lanes beyond G r idle), consecutive lanes reading consecutive
// entries of a column.  The groups' sums meet by warp shuffles, the warps' by shared
// memory, both in a fixed order.
//
// FP64 form: one matrix, the stored FP64 blocks (free space, reaction, self terms).
// Precision form (MIX): the blocks without reaction entries in complex64 with their
// self terms taken out, multiplied with x rounded to complex64 (FP32 products and
// sums); the blocks that hold reaction entries as FP64 copies, and the self terms as
// an FP64 diagonal, with the FP64 x; the parts are added in FP64.
struct NearRowPart {
    const int64_t* off;   // per leaf: first value of its matrix
    const int* jptr;      // per leaf: column range [jptr[T], jptr[T + 1])
    const int* j;         // sorted source position of each column
};

__device__ __forceinline__ void near_fma(cd& acc, const cd& v, const cd& x) { cfma(acc, v, x); }
__device__ __forceinline__ void near_fma(float2& acc, const float2& v, const float2& x) {
    acc.x = fmaf(v.x, x.x, acc.x);
    acc.x = fmaf(-v.y, x.y, acc.x);
    acc.y = fmaf(v.x, x.y, acc.y);
    acc.y = fmaf(v.y, x.x, acc.y);
}

// acc[q] += sum over the columns [ca, cb) of the leaf's matrix taken by this lane group, for
// the right-hand sides q < ncb (x + q n): each stored entry is read once for all of them, and
// every right-hand side's sum runs in the order of the single-column sum (four partial sums)
template <int CB, typename V, typename X, typename A>
__device__ __forceinline__ void near_row_sum(const V* __restrict__ val, const NearRowPart& P, int leaf, int nT, int i,
                                             int g, int G, int ca, int cb, const X* __restrict__ x, int64_t n,
                                             int ncb, A (&acc)[CB]) {
    const int c0 = P.jptr[leaf];
    const V* v = val + P.off[leaf] + i;
    A a1[CB], a2[CB], a3[CB];
#pragma unroll
    for (int q = 0; q < CB; ++q) { a1[q] = A{}; a2[q] = A{}; a3[q] = A{}; }
    int c = ca + g;
    // four columns in flight per lane
    for (; c + 3 * G < cb; c += 4 * G) {
        const V v0 = v[(int64_t)(c - c0) * nT], v1 = v[(int64_t)(c + G - c0) * nT];
        const V v2 = v[(int64_t)(c + 2 * G - c0) * nT], v3 = v[(int64_t)(c + 3 * G - c0) * nT];
        const int j0 = P.j[c], j1 = P.j[c + G], j2 = P.j[c + 2 * G], j3 = P.j[c + 3 * G];
#pragma unroll
        for (int q = 0; q < CB; ++q) {
            if (q < ncb) {
                const X* xq = x + q * n;
                near_fma(acc[q], v0, xq[j0]);
                near_fma(a1[q], v1, xq[j1]);
                near_fma(a2[q], v2, xq[j2]);
                near_fma(a3[q], v3, xq[j3]);
            }
        }
    }
    for (; c < cb; c += G) {
        const V vc = v[(int64_t)(c - c0) * nT];
        const int jc = P.j[c];
#pragma unroll
        for (int q = 0; q < CB; ++q)
            if (q < ncb) near_fma(acc[q], vc, x[q * n + jc]);
    }
#pragma unroll
    for (int q = 0; q < CB; ++q) {
        acc[q].x += a1[q].x; acc[q].y += a1[q].y;
        a2[q].x += a3[q].x; a2[q].y += a3[q].y;
        acc[q].x += a2[q].x; acc[q].y += a2[q].y;
    }
}
template <int NW>
__device__ __forceinline__ void share(const NearRowPart& P, int leaf, int w, int* ca, int* cb) {
    const int c0 = P.jptr[leaf], nj = P.jptr[leaf + 1] - c0;
    *ca = c0 + (int)(((int64_t)nj * w) / NW);
    *cb = c0 + (int)(((int64_t)nj * (w + 1)) / NW);
}

// NW warps per leaf.  With few leaves (fewer than two waves of single-warp leaves) several
// warps share a leaf so that enough loads are in flight: 2 in the FP64 form (bound by the
// FP64 pipe; fewer warps per leaf keep the fixed cost of the reductions small against the
// FMAs), 4 in the precision form (bound by memory).  With many leaves one warp per leaf
// keeps four times as many leaves in flight per SM and needs no barrier.  In the precision
// form the FP32 part is reduced in FP32 and converted once per row, and the FP64 part is
// skipped for the leaves without reaction columns.
template <bool MIX, int NW, int CB>
__device__ __forceinline__ void near_leaf_cta(int leaf, int leaf0, const int* __restrict__ box_begin,
                                              const int* __restrict__ box_end, const NearRowPart& P64,
                                              const cd* __restrict__ val64, const NearRowPart& P32,
                                              const float2* __restrict__ val32, const cd* __restrict__ diag,
                                              const cd* __restrict__ x, const float2* __restrict__ x32,
                                              cd* __restrict__ y, int64_t n, int nrhs) {
    __shared__ cd part[NW][32];
    __shared__ float2 part32[MIX ? NW : 1][32];
    const int w = NW == 1 ? 0 : (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int tb = box_begin[leaf0 + leaf], nT = box_end[leaf0 + leaf] - tb;
    const bool has64 = !MIX || P64.jptr[leaf + 1] > P64.jptr[leaf];   // the same for the whole CTA
    int a64, b64, a32 = 0, b32 = 0;
    share<NW>(P64, leaf, w, &a64, &b64);
    if (MIX) share<NW>(P32, leaf, w, &a32, &b32);
    for (int col0 = 0; col0 < nrhs; col0 += CB) {   // CB right-hand sides per pass over the entries
        const int ncb = min(CB, nrhs - col0);
        for (int i0 = 0; i0 < nT; i0 += 32) {
            const int r = min(32, nT - i0), G = 32 / r;
            const int i = i0 + lane % r, g = lane / r;
            cd acc[CB];
            float2 s32[CB];
#pragma unroll
            for (int q = 0; q < CB; ++q) { acc[q] = mk(0.0, 0.0); s32[q] = make_float2(0.f, 0.f); }
            if (g < G) {
                if (has64) near_row_sum<CB>(val64, P64, leaf, nT, i, g, G, a64, b64, x + (int64_t)col0 * n, n, ncb, acc);
                if (MIX)
                    near_row_sum<CB>(val32, P32, leaf, nT, i, g, G, a32, b32, x32 + (int64_t)col0 * n, n, ncb, s32);
            }
#pragma unroll
            for (int q = 0; q < CB; ++q) {
                if (q >= ncb) break;
                const int col = col0 + q;
                const cd* xc = x + (int64_t)col * n;
                for (int gg = 1; gg < G; ++gg) {
                    const int src = (lane + gg * r) & 31;
                    if (has64) {
                        const double ox = __shfl_sync(0xffffffffu, acc[q].x, src);
                        const double oy = __shfl_sync(0xffffffffu, acc[q].y, src);
                        if (lane < r) { acc[q].x += ox; acc[q].y += oy; }
                    }
                    if (MIX) {
                        const float ox = __shfl_sync(0xffffffffu, s32[q].x, src);
                        const float oy = __shfl_sync(0xffffffffu, s32[q].y, src);
                        if (lane < r) { s32[q].x += ox; s32[q].y += oy; }
                    }
                }
                if (NW == 1) {   // one warp per leaf: no exchange between warps
                    if (lane < r) {
                        cd t = has64 ? acc[q] : mk(0.0, 0.0);
                        if (MIX) {
                            t.x += (double)s32[q].x;
                            t.y += (double)s32[q].y;
                            cfma(t, diag[tb + i], xc[tb + i]);
                        }
                        y[(int64_t)col * n + tb + i] += t;
                    }
                    continue;
                }
                if (lane < r) {
                    if (has64) part[w][lane] = acc[q];
                    if (MIX) part32[w][lane] = s32[q];
                }
                __syncthreads();
                if (w == 0 && lane < r) {
                    cd t = mk(0.0, 0.0);
                    if (has64) {
                        t = part[0][lane];
                        for (int k = 1; k < NW; ++k) t += part[k][lane];
                    }
                    if (MIX) {
                        float2 u = part32[0][lane];
                        for (int k = 1; k < NW; ++k) { u.x += part32[k][lane].x; u.y += part32[k][lane].y; }
                        t.x += (double)u.x;
                        t.y += (double)u.y;
                        cfma(t, diag[tb + i], xc[tb + i]);
                    }
                    y[(int64_t)col * n + tb + i] += t;
                }
                __syncthreads();
            }
        }
    }
}
#define NEAR_WARPS_64 2
#define NEAR_WARPS_MIX 4
// CB: right-hand sides per pass over the stored entries (1, or 4 for a block right-hand side)
template <bool MIX, int NW, int CB>
__global__ void __launch_bounds__(32 * NW) k_near_leaf(int leaf0, const int* __restrict__ box_begin,
                                                       const int* __restrict__ box_end, NearRowPart P64,
                                                       const cd* __restrict__ val64, NearRowPart P32,
                                                       const float2* __restrict__ val32, const cd* __restrict__ diag,
                                                       const cd* __restrict__ x, const float2* __restrict__ x32,
                                                       cd* __restrict__ y, int64_t n, int nrhs) {
    near_leaf_cta<MIX, NW, CB>(blockIdx.x, leaf0, box_begin, box_end, P64, val64, P32, val32, diag, x, x32, y, n, nrhs);
}
// one warp per leaf, four warps per CTA
template <bool MIX, int CB>
__global__ void __launch_bounds__(128) k_near_leaf_w(int nleaf, int leaf0, const int* __restrict__ box_begin,
                                                     const int* __restrict__ box_end, NearRowPart P64,
                                                     const cd* __restrict__ val64, NearRowPart P32,
                                                     const float2* __restrict__ val32, const cd* __restrict__ diag,
                                                     const cd* __restrict__ x, const float2* __restrict__ x32,
                                                     cd* __restrict__ y, int64_t n, int nrhs) {
    const int leaf = (int)(blockIdx.x * 4 + (threadIdx.x >> 5));
    if (leaf >= nleaf) return;   // whole warps: the single-warp path has no block barrier
    near_leaf_cta<MIX, 1, CB>(leaf, leaf0, box_begin, box_end, P64, val64, P32, val32, diag, x, x32, y, n, nrhs);
}
// leaves from which one warp per leaf fills two waves of the GPU (152 SMs x 64 warps x 2)
#define NEAR_WARP_PER_LEAF_MIN (152 * 64 * 2)
// x rounded to complex64 (the precision form's FP32 near-field products)
__global__ void k_round_x32(const cd* __restrict__ x, float2* __restrict__ x32, int64_t tot) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x)
        x32[q] = make_float2((float)x[q].x, (float)x[q].y);
}

// one block copied into the precision form's stores
struct NearCopy {
    int64_t src;    // offset in the FP64 blocks
    int64_t dst;    // offset in the FP32 or FP64 store
    int nT, nS;
    int self;       // 1: block (T, T) going to FP32: its diagonal moves to the FP64 diagonal
    int to32;       // 1: FP32 store, 0: FP64 store
    int tb;         // first sorted position of T
};
__global__ void k_near_repack(const NearCopy* __restrict__ cp, const cd* __restrict__ val, float2* __restrict__ v32,
                              cd* __restrict__ v64, cd* __restrict__ diag) {
    const NearCopy c = cp[blockIdx.x];
    const int ne = c.nT * c.nS;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const cd v = val[c.src + e];
        if (!c.to32) {
            v64[c.dst + e] = v;
            continue;
        }
        const int i = e % c.nT, j = e / c.nT;
        if (c.self && i == j) {
            diag[c.tb + i] = v;
            v32[c.dst + e] = make_float2(0.f, 0.f);
        } else {
            v32[c.dst + e] = make_float2((float)v.x, (float)v.y);
        }
    }
}

void near_build(lfmm_geometry_s* g) {
    TreeHost& t = g->tree;
    const int D = t.D;
    g->leaf0 = t.level_start[D];
    g->nleaf = t.level_start[D + 1] - g->leaf0;
    // blocks per target leaf: union of free-space and reaction near lists
    std::vector<int> blk_tgt, blk_src, nb_ptr(g->nleaf + 1, 0);
    std::vector<unsigned char> blk_free, blk_react;
    std::vector<int64_t> blk_off;
    std::vector<NearTask> tasks;
    std::vector<int> task_comp;
    int64_t off = 0, work = 0;
    for (int li = 0; li < g->nleaf; ++li) {
        const int T = g->leaf0 + li;
        if (g->n_src < g->n) {   // field geometry: only the rows of field points are needed
            bool has_field = false;
            for (int q = t.box_begin[T]; q < t.box_end[T] && !has_field; ++q) has_field = t.perm[q] >= g->n_src;
            if (!has_field) {
                nb_ptr[li + 1] = (int)blk_tgt.size();
                continue;
            }
        }
        std::vector<int> srcs;
        for (int k = t.ufree_ptr[T]; k < t.ufree_ptr[T + 1]; ++k) srcs.push_back(t.ufree_idx[k]);
        for (int k = t.ureact_ptr[T]; k < t.ureact_ptr[T + 1]; ++k) srcs.push_back(t.ureact_idx[k]);
        std::sort(srcs.begin(), srcs.end());
        srcs.erase(std::unique(srcs.begin(), srcs.end()), srcs.end());
        const int nT = t.box_end[T] - t.box_begin[T];
        for (int S : srcs) {
            int bi = (int)blk_tgt.size();
            blk_tgt.push_back(T);
            blk_src.push_back(S);
            bool fr = false;
            for (int k = t.ufree_ptr[T]; k < t.ufree_ptr[T + 1]; ++k) fr |= (t.ufree_idx[k] == S);
            blk_free.push_back(fr ? 1 : 0);
            blk_off.push_back(off);
            const int nS = t.box_end[S] - t.box_begin[S];
            const int c0 = (int)task_comp.size();
            for (int k = t.ureact_ptr[T]; k < t.ureact_ptr[T + 1]; ++k)
                if (t.ureact_idx[k] == S) task_comp.push_back(t.ureact_comp[k]);
            const bool re = (int)task_comp.size() > c0;
            if (re) {
                tasks.push_back(NearTask{bi, c0, (int)task_comp.size(), work});
                work += (int64_t)nT * nS;
            }
            blk_react.push_back(re ? 1 : 0);
            off += (int64_t)nT * nS;
        }
        nb_ptr[li + 1] = (int)blk_tgt.size();
    }
    g->n_blocks = (int)blk_tgt.size();
    g->nb_nnz = off;
    int* d_bt = dupload(g, blk_tgt);
    g->d_nb_src = dupload(g, blk_src);
    g->d_nb_off = dupload(g, blk_off);
    g->d_nb_ptr = dupload(g, nb_ptr);
    unsigned char* d_bf = dupload(g, blk_free);
    g->d_nb_val = dalloc<cd>(g, (size_t)off);
    // each leaf's blocks as one matrix: column -> sorted source position
    {
        std::vector<int> jptr(g->nleaf + 1, 0), jl;
        std::vector<int64_t> loff(g->nleaf, 0);
        for (int li = 0; li < g->nleaf; ++li) {
            loff[li] = nb_ptr[li] < nb_ptr[li + 1] ? blk_off[nb_ptr[li]] : 0;
            for (int k = nb_ptr[li]; k < nb_ptr[li + 1]; ++k)
                for (int p = t.box_begin[blk_src[k]]; p < t.box_end[blk_src[k]]; ++p) jl.push_back(p);
            jptr[li + 1] = (int)jl.size();
        }
        g->d_nl_jptr = dupload(g, jptr);
        g->d_nl_j = dupload(g, jl);
        g->d_nl_off = dupload(g, loff);
    }
    g->nb_ptr_host = nb_ptr;
    g->nb_src_host = blk_src;
    g->nb_off_host = blk_off;
    g->nb_react_host = blk_react;
    std::vector<double> compH(t.comps.size());
    for (size_t c = 0; c < t.comps.size(); ++c) compH[c] = t.comps[c].Hc;
    double* d_compH = dupload(g, compH);
    if (g->n_blocks > 0) {
        k_near_free<<<g->n_blocks, 128>>>(g->m, d_bt, g->d_nb_src, g->d_nb_off, d_bf, g->d_box_begin,
                                          g->d_box_end, g->d_box_layer, g->d_x, g->d_y, g->d_w, g->d_nx, g->d_ny,
                                          g->d_nb_val);
        cuda_check(cudaGetLastError(), "k_near_free");
    }
    if (!tasks.empty()) {
        NearTask* d_tasks = dupload(g, tasks);
        int* d_task_comp = dupload(g, task_comp);
        int threads = 256;
        int64_t warps_needed = work;
        int64_t blocks = std::min<int64_t>((warps_needed * 32 + threads - 1) / threads, 152 * 64);
        k_near_react<<<(int)blocks, threads>>>(g->m, g->quad, d_tasks, (int)tasks.size(), work, d_task_comp, d_bt,
                                               g->d_nb_src, g->d_nb_off, g->d_comp, d_compH, g->d_box_begin,
                                               g->d_box_end, g->d_x, g->d_y, g->d_w, g->d_nx, g->d_ny,
                                               g->d_nb_val);
        cuda_check(cudaGetLastError(), "k_near_react");
    }
    cuda_check(cudaStreamSynchronize(cudaStreamPerThread), "near_build");
}

// The precision form's near field (built on its first use): blocks without reaction
// entries in complex64 with the self terms moved to an FP64 diagonal, blocks with
// reaction entries (Sommerfeld quadrature near interfaces) kept in FP64.
static void near_mixed_build(lfmm_geometry_s* g) {
    const TreeHost& t = g->tree;
    const int nleaf = g->nleaf;
    std::vector<NearCopy> cps;
    std::vector<int> jp32(nleaf + 1, 0), jp64(nleaf + 1, 0), j32, j64;
    std::vector<int64_t> o32(nleaf, 0), o64(nleaf, 0);
    int64_t n32 = 0, n64 = 0;
    for (int li = 0; li < nleaf; ++li) {
        const int T = g->leaf0 + li;
        const int tb = t.box_begin[T], nT = t.box_end[T] - tb;
        o32[li] = n32;
        o64[li] = n64;
        for (int k = g->nb_ptr_host[li]; k < g->nb_ptr_host[li + 1]; ++k) {
            const int S = g->nb_src_host[k];
            const int nS = t.box_end[S] - t.box_begin[S];
            const bool to32 = g->nb_react_host[k] == 0;
            NearCopy c{g->nb_off_host[k], to32 ? n32 : n64, nT, nS, (to32 && S == T) ? 1 : 0, to32 ? 1 : 0, tb};
            cps.push_back(c);
            std::vector<int>& jl = to32 ? j32 : j64;
            for (int p = t.box_begin[S]; p < t.box_end[S]; ++p) jl.push_back(p);
            (to32 ? n32 : n64) += (int64_t)nT * nS;
        }
        jp32[li + 1] = (int)j32.size();
        jp64[li + 1] = (int)j64.size();
    }
    g->d_nl_jptr32 = dupload(g, jp32);
    g->d_nl_j32 = dupload(g, j32);
    g->d_nl_off32 = dupload(g, o32);
    g->d_nl_jptr64r = dupload(g, jp64);
    g->d_nl_j64r = dupload(g, j64);
    g->d_nl_off64r = dupload(g, o64);
    g->d_nv32 = dalloc<float2>(g, (size_t)n32);
    g->d_nv64r = dalloc<cd>(g, (size_t)n64);
    g->d_ndiag = dalloc<cd>(g, (size_t)g->n);
    g->near32_nnz = n32;
    g->near64r_nnz = n64;
    cuda_check(cudaMemsetAsync(g->d_ndiag, 0, sizeof(cd) * g->n, cudaStreamPerThread), "memset diag");
    if (!cps.empty()) {
        NearCopy* d_cps = dupload(g, cps);
        k_near_repack<<<(int)cps.size(), 128, 0, cudaStreamPerThread>>>(d_cps, g->d_nb_val, g->d_nv32, g->d_nv64r,
                                                                        g->d_ndiag);
        cuda_check(cudaGetLastError(), "k_near_repack");
    }
    cuda_check(cudaStreamSynchronize(cudaStreamPerThread), "near_mixed_build");
    g->near32_ready = true;
}

// Several geometries' FP64 near fields in one launch: four leaves (warps) per CTA, the CTAs
// of each geometry consecutive; a CTA finds its geometry by binary search over the prefix.
struct NearJob {
    int nleaf, leaf0;
    const int *box_begin, *box_end;
    NearRowPart P64;
    const cd* val64;
    const cd* x;
    cd* y;
    int64_t n;
    int nrhs;
};
template <int CB>
__global__ void __launch_bounds__(32 * NEAR_WARPS_64) k_near_leaf_multi(const NearJob* __restrict__ jobs,
                                                                     const int* __restrict__ prefix, int njobs) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const NearJob& J = jobs[lo];
    near_leaf_cta<false, NEAR_WARPS_64, CB>((int)blockIdx.x - prefix[lo], J.leaf0, J.box_begin, J.box_end, J.P64, J.val64, J.P64,
                         nullptr, nullptr, J.x, nullptr, J.y, J.n, J.nrhs);
}

void near_apply_batch(const std::vector<BatchOp>& ops, cudaStream_t s) {
    std::vector<NearJob> jobs;
    std::vector<int> prefix(1, 0);
    for (const BatchOp& op : ops) {
        lfmm_geometry_s* g = op.g;
        if (g->nleaf >= NEAR_WARP_PER_LEAF_MIN) {   // as near_apply: its own warp-per-leaf launch (same sums)
            const NearRowPart p64{g->d_nl_off, g->d_nl_jptr, g->d_nl_j};
            if (op.nrhs > 1)
                k_near_leaf_w<false, 4><<<(g->nleaf + 3) / 4, 128, 0, s>>>(g->nleaf, g->leaf0, g->d_box_begin,
                                                                       g->d_box_end, p64, g->d_nb_val, p64, nullptr,
                                                                       nullptr, op.x, nullptr, op.y, g->n, op.nrhs);
            else
                k_near_leaf_w<false, 1><<<(g->nleaf + 3) / 4, 128, 0, s>>>(g->nleaf, g->leaf0, g->d_box_begin,
                                                                       g->d_box_end, p64, g->d_nb_val, p64, nullptr,
                                                                       nullptr, op.x, nullptr, op.y, g->n, op.nrhs);
            cuda_check(cudaGetLastError(), "k_near_leaf_w");
            continue;
        }
        jobs.push_back(NearJob{g->nleaf, g->leaf0, g->d_box_begin, g->d_box_end,
                               NearRowPart{g->d_nl_off, g->d_nl_jptr, g->d_nl_j}, g->d_nb_val, op.x, op.y, g->n,
                               op.nrhs});
        prefix.push_back(prefix.back() + g->nleaf);
    }
    if (prefix.back() == 0) return;
    JobTables t;
    const size_t oj = t.add(jobs.data(), sizeof(NearJob) * jobs.size());
    const size_t op = t.add(prefix.data(), sizeof(int) * prefix.size());
    t.upload(s);
    int maxr = 1;
    for (const NearJob& J : jobs) maxr = std::max(maxr, J.nrhs);
    if (maxr > 1)
        k_near_leaf_multi<4><<<prefix.back(), 32 * NEAR_WARPS_64, 0, s>>>(t.at<NearJob>(oj), t.at<int>(op),
                                                                          (int)jobs.size());
    else
        k_near_leaf_multi<1><<<prefix.back(), 32 * NEAR_WARPS_64, 0, s>>>(t.at<NearJob>(oj), t.at<int>(op),
                                                                          (int)jobs.size());
    cudaError_t e = cudaGetLastError();
    t.release(s);
    cuda_check(e, "k_near_leaf_multi");
}

void near_apply(lfmm_geometry_s* g, const cd* x_sorted, cd* y_sorted, int nrhs, cudaStream_t s, bool mixed) {
    if (g->nleaf == 0) return;
    if (mixed && !g->near32_ready) near_mixed_build(g);
    prof_begin(g, ST_NEAR, s);
    if (mixed) {
        const int64_t tot = g->n * nrhs;
        if (g->near_x32_cap < tot) {
            dev_release_now(g->d_near_x32);
            g->d_near_x32 = nullptr;
            g->d_near_x32 = (float2*)dev_alloc_ready(sizeof(float2) * tot, "near x32");
            g->near_x32_cap = tot;
        }
        k_round_x32<<<(int)std::min<int64_t>((tot + 255) / 256, 152 * 16), 256, 0, s>>>(x_sorted, g->d_near_x32, tot);
        cuda_check(cudaGetLastError(), "k_round_x32");
        ++g->n_launches;
        const NearRowPart p64{g->d_nl_off64r, g->d_nl_jptr64r, g->d_nl_j64r};
        const NearRowPart p32{g->d_nl_off32, g->d_nl_jptr32, g->d_nl_j32};
        if (g->nleaf >= NEAR_WARP_PER_LEAF_MIN) {
            if (nrhs > 1)
                k_near_leaf_w<true, 4><<<(g->nleaf + 3) / 4, 128, 0, s>>>(g->nleaf, g->leaf0, g->d_box_begin,
                                                                       g->d_box_end, p64, g->d_nv64r, p32, g->d_nv32,
                                                                       g->d_ndiag, x_sorted, g->d_near_x32, y_sorted,
                                                                       g->n, nrhs);
            else
                k_near_leaf_w<true, 1><<<(g->nleaf + 3) / 4, 128, 0, s>>>(g->nleaf, g->leaf0, g->d_box_begin,
                                                                       g->d_box_end, p64, g->d_nv64r, p32, g->d_nv32,
                                                                       g->d_ndiag, x_sorted, g->d_near_x32, y_sorted,
                                                                       g->n, nrhs);
        } else if (nrhs > 1) {
            k_near_leaf<true, NEAR_WARPS_MIX, 4><<<g->nleaf, 32 * NEAR_WARPS_MIX, 0, s>>>(
                g->leaf0, g->d_box_begin, g->d_box_end, p64, g->d_nv64r, p32, g->d_nv32, g->d_ndiag, x_sorted,
                g->d_near_x32, y_sorted, g->n, nrhs);
        } else {
            k_near_leaf<true, NEAR_WARPS_MIX, 1><<<g->nleaf, 32 * NEAR_WARPS_MIX, 0, s>>>(
                g->leaf0, g->d_box_begin, g->d_box_end, p64, g->d_nv64r, p32, g->d_nv32, g->d_ndiag, x_sorted,
                g->d_near_x32, y_sorted, g->n, nrhs);
        }
    } else {
        const NearRowPart p64{g->d_nl_off, g->d_nl_jptr, g->d_nl_j};
        if (g->nleaf >= NEAR_WARP_PER_LEAF_MIN) {
            if (nrhs > 1)
                k_near_leaf_w<false, 4><<<(g->nleaf + 3) / 4, 128, 0, s>>>(g->nleaf, g->leaf0, g->d_box_begin,
                                                                        g->d_box_end, p64, g->d_nb_val, p64, nullptr,
                                                                        nullptr, x_sorted, nullptr, y_sorted, g->n,
                                                                        nrhs);
            else
                k_near_leaf_w<false, 1><<<(g->nleaf + 3) / 4, 128, 0, s>>>(g->nleaf, g->leaf0, g->d_box_begin,
                                                                        g->d_box_end, p64, g->d_nb_val, p64, nullptr,
                                                                        nullptr, x_sorted, nullptr, y_sorted, g->n,
                                                                        nrhs);
        } else if (nrhs > 1) {
            k_near_leaf<false, NEAR_WARPS_64, 4><<<g->nleaf, 32 * NEAR_WARPS_64, 0, s>>>(
                g->leaf0, g->d_box_begin, g->d_box_end, p64, g->d_nb_val, p64, nullptr, nullptr, x_sorted, nullptr,
                y_sorted, g->n, nrhs);
        } else {
            k_near_leaf<false, NEAR_WARPS_64, 1><<<g->nleaf, 32 * NEAR_WARPS_64, 0, s>>>(
                g->leaf0, g->d_box_begin, g->d_box_end, p64, g->d_nb_val, p64, nullptr, nullptr, x_sorted, nullptr,
                y_sorted, g->n, nrhs);
        }
    }
    cuda_check(cudaGetLastError(), "k_near_leaf");
    ++g->n_launches;
    prof_end(g, ST_NEAR, s);
}

}  // namespace lfmm
