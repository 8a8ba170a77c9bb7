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

struct NearTask {   // one (block, component) reaction task
    int blk;        // block index
    int comp;
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
            if (pi == pj) {
                out = self_entry(k, pw[pi], cf);
            } else {
                out = pw[pj] * free_kernel(k, px[pj] - px[pi], py[pj] - py[pi], cf, cf ? nx[pj] : 0.0,
                                           cf ? ny[pj] : 0.0);
            }
        }
        v[(int64_t)j * nT + i] = out;
    }
}

// reaction entries: one warp per (task, entry)
__global__ void k_near_react(MediumDev m, QuadRule q, const NearTask* __restrict__ tasks, int ntask,
                             int64_t nwork, const int* __restrict__ blk_tgt, const int* __restrict__ blk_src,
                             const int64_t* __restrict__ blk_off, const int* __restrict__ comp,
                             const double* __restrict__ comp_H, const int* __restrict__ box_begin,
                             const int* __restrict__ box_end, const double* __restrict__ px,
                             const double* __restrict__ py, const double* __restrict__ pw,
                             const double* __restrict__ nx, const double* __restrict__ ny, cd* __restrict__ val) {
    const bool cf = nx != nullptr;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wk = warp; wk < nwork; wk += nwarps) {
        // locate the task by binary search on first
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
        const int c = tk.comp;
        const int ls = comp[4 * c], a = comp[4 * c + 1], lt = comp[4 * c + 2], b = comp[4 * c + 3];
        const int pi = tb + i, pj = sb + j;
        const double X = px[pj] - px[pi];
        const double hs = (a == 0) ? (py[pj] - m.yint[ls]) : (m.yint[ls - 1] - py[pj]);
        const double ht = (b == 0) ? (m.yint[lt - 1] - py[pi]) : (py[pi] - m.yint[lt]);
        cd K;
        if (cf) {
            cd gk[3];
            react_kernel_grad_warp(m, q, ls, a, lt, b, comp_H[c], X, hs, ht, gk);
            K = react_cf_combine(gk, a, m.k[ls], nx[pj], ny[pj]);
        } else {
            K = react_kernel_warp(m, q, ls, a, lt, b, comp_H[c], X, hs, ht);
        }
        if ((threadIdx.x & 31) == 0) {
            cd* dst = val + blk_off[tk.blk] + (int64_t)j * nT + i;
            double wj = pw[pj];
            atomicAdd(&dst->x, wj * K.x);
            atomicAdd(&dst->y, wj * K.y);
        }
    }
}

// y_T += sum_S B_{TS} x_S for all target leaves (one CTA per leaf)
__global__ void __launch_bounds__(128) k_near_apply(const int* __restrict__ nb_ptr, const int* __restrict__ nb_src,
                                                    const int64_t* __restrict__ nb_off, const cd* __restrict__ val,
                                                    const int* __restrict__ box_begin, const int* __restrict__ box_end,
                                                    int leaf0, const cd* __restrict__ x, cd* __restrict__ y,
                                                    int64_t n, int nrhs) {
    __shared__ cd part[128];
    const int T = leaf0 + blockIdx.x;
    const int tb = box_begin[T], nT = box_end[T] - tb;
    for (int col = 0; col < nrhs; ++col) {
        const cd* xc = x + (int64_t)col * n;
        for (int i0 = 0; i0 < nT; i0 += blockDim.x) {
            const int nTi = min(nT - i0, (int)blockDim.x);
            const int Gi = (nTi >= (int)blockDim.x) ? 1 : (int)blockDim.x / nTi;
            const int i = i0 + (threadIdx.x % nTi);
            const int g = threadIdx.x / nTi;
            cd acc = mk(0.0, 0.0);
            if (g < Gi) {
                for (int k = nb_ptr[blockIdx.x]; k < nb_ptr[blockIdx.x + 1]; ++k) {
                    const int S = nb_src[k];
                    const int sb = box_begin[S], nS = box_end[S] - sb;
                    const cd* v = val + nb_off[k];
                    for (int j = g; j < nS; j += Gi) cfma(acc, v[(int64_t)j * nT + i], xc[sb + j]);
                }
            }
            part[threadIdx.x] = acc;
            __syncthreads();
            if (threadIdx.x < nTi) {
                cd s = mk(0.0, 0.0);
                for (int gg = 0; gg < Gi; ++gg) s += part[gg * nTi + threadIdx.x];
                y[(int64_t)col * n + tb + i0 + threadIdx.x] += s;
            }
            __syncthreads();
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
    std::vector<unsigned char> blk_free;
    std::vector<int64_t> blk_off;
    std::vector<NearTask> tasks;
    int64_t off = 0, work = 0;
    for (int li = 0; li < g->nleaf; ++li) {
        const int T = g->leaf0 + li;
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
            for (int k = t.ureact_ptr[T]; k < t.ureact_ptr[T + 1]; ++k) {
                if (t.ureact_idx[k] != S) continue;
                tasks.push_back(NearTask{bi, t.ureact_comp[k], work});
                work += (int64_t)nT * nS;
            }
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
        int threads = 256;
        int64_t warps_needed = work;
        int64_t blocks = std::min<int64_t>((warps_needed * 32 + threads - 1) / threads, 152 * 64);
        k_near_react<<<(int)blocks, threads>>>(g->m, g->quad, d_tasks, (int)tasks.size(), work, d_bt,
                                               g->d_nb_src, g->d_nb_off, g->d_comp, d_compH, g->d_box_begin,
                                               g->d_box_end, g->d_x, g->d_y, g->d_w, g->d_nx, g->d_ny,
                                               g->d_nb_val);
        cuda_check(cudaGetLastError(), "k_near_react");
    }
    cuda_check(cudaStreamSynchronize(cudaStreamPerThread), "near_build");
}

void near_apply(lfmm_geometry_s* g, const cd* x_sorted, cd* y_sorted, int nrhs, cudaStream_t s) {
    if (g->nleaf == 0) return;
    prof_begin(g, ST_NEAR, s);
    k_near_apply<<<g->nleaf, 128, 0, s>>>(g->d_nb_ptr, g->d_nb_src, g->d_nb_off, g->d_nb_val, g->d_box_begin,
                                          g->d_box_end, g->leaf0, x_sorted, y_sorted, g->n, nrhs);
    cuda_check(cudaGetLastError(), "k_near_apply");
    ++g->n_launches;
    prof_end(g, ST_NEAR, s);
}

}  // namespace lfmm
