// precond.cu -- overlapping domain-decomposition preconditioner (Sec. 4.2).
//
// For every leaf B of every layer's tree the local system P_B of eq.
// localmatix is assembled on the points J of B and of its neighbour leaves
// (the leaf's free-space near list), with the free-space entries
// |Gamma_j| G^f(c_j, c_i) off the diagonal and the self terms I^s on it (the
// reaction part is left out, as in the paper's K~); in the combined-field form
// the same entries of that operator (devmath.cuh: free_kernel, self_entry).
// Only the rows of P_B^{-1} that belong to B's own points are kept
// (restriction Q_B), so
//   P^{-1} v = sum_B S_B Q_B P_B^{-1} R_B v
// is one gather, one small dense product and one scatter per leaf.  The rows
// are obtained from an LU factorisation with partial pivoting of P_B^T.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "geometry.h"

namespace lfmm {

// one CTA per leaf: assemble A = P_B^T, factor, solve A X = E_own, store W (column-major: W[b * s + i])
__global__ void __launch_bounds__(256) k_pc_setup(MediumDev m, const int* __restrict__ pc_ptr,
                                                  const int* __restrict__ pc_idx, const int* __restrict__ own_pos,
                                                  const int* __restrict__ own_cnt, const int64_t* __restrict__ aoff,
                                                  const int64_t* __restrict__ woff, const int* __restrict__ layer_of_leaf,
                                                  const double* __restrict__ px, const double* __restrict__ py,
                                                  const double* __restrict__ pw, const double* __restrict__ nx,
                                                  const double* __restrict__ ny, cd* __restrict__ Ascr,
                                                  int* __restrict__ pivscr, cd* __restrict__ W) {
    const int B = blockIdx.x;
    const int jb = pc_ptr[B], q = pc_ptr[B + 1] - jb;
    const int s = own_cnt[B], o0 = own_pos[B];
    const double k = m.k[layer_of_leaf[B]];
    cd* A = Ascr + aoff[B];            // row-major q x q
    int* piv = pivscr + jb;
    __shared__ double red_v[256];
    __shared__ int red_i[256];
    // A[a][b] = P[b][a]: P[i][j] = w_j G(c_j, c_i) (i != j), I^s_i (i == j)
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
        int a = e / q, b = e % q;
        int i = pc_idx[jb + b], j = pc_idx[jb + a];   // P[i=b][j=a]
        const bool cf = nx != nullptr;
        A[e] = (a == b) ? self_entry(k, pw[i], cf)
                        : pw[j] * free_kernel(k, px[j] - px[i], py[j] - py[i], cf, cf ? nx[j] : 0.0, cf ? ny[j] : 0.0);
    }
    __syncthreads();
    // LU with partial pivoting
    for (int c = 0; c < q; ++c) {
        double best = -1.0;
        int bi = c;
        for (int r = c + threadIdx.x; r < q; r += blockDim.x) {
            double v = absc(A[(int64_t)r * q + c]);
            if (v > best) { best = v; bi = r; }
        }
        red_v[threadIdx.x] = best;
        red_i[threadIdx.x] = bi;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o && red_v[threadIdx.x + o] > red_v[threadIdx.x]) {
                red_v[threadIdx.x] = red_v[threadIdx.x + o];
                red_i[threadIdx.x] = red_i[threadIdx.x + o];
            }
            __syncthreads();
        }
        const int pr = red_i[0];
        __syncthreads();
        if (threadIdx.x == 0) piv[c] = pr;
        if (pr != c)
            for (int jj = threadIdx.x; jj < q; jj += blockDim.x) {
                cd t = A[(int64_t)c * q + jj];
                A[(int64_t)c * q + jj] = A[(int64_t)pr * q + jj];
                A[(int64_t)pr * q + jj] = t;
            }
        __syncthreads();
        const cd inv = cinv(A[(int64_t)c * q + c]);
        for (int r = c + 1 + threadIdx.x; r < q; r += blockDim.x) A[(int64_t)r * q + c] = A[(int64_t)r * q + c] * inv;
        __syncthreads();
        const int rem = q - c - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            int r = c + 1 + e / rem, jj = c + 1 + e % rem;
            cfma(A[(int64_t)r * q + jj], -A[(int64_t)r * q + c], A[(int64_t)c * q + jj]);
        }
        __syncthreads();
    }
    // solve A X = E for the own columns; thread t handles own column t
    cd* Wb = W + woff[B];
    for (int t = threadIdx.x; t < s; t += blockDim.x) {
        // X column stored in W as W[b * s + t]
        for (int b = 0; b < q; ++b) Wb[(int64_t)b * s + t] = mk(0.0, 0.0);
        Wb[(int64_t)(o0 + t) * s + t] = mk(1.0, 0.0);
        for (int c = 0; c < q; ++c) {   // apply row swaps
            int pr = piv[c];
            if (pr != c) {
                cd tmp = Wb[(int64_t)c * s + t];
                Wb[(int64_t)c * s + t] = Wb[(int64_t)pr * s + t];
                Wb[(int64_t)pr * s + t] = tmp;
            }
        }
        for (int r = 0; r < q; ++r) {   // L y = P e (unit lower)
            cd acc = Wb[(int64_t)r * s + t];
            for (int c = 0; c < r; ++c) cfma(acc, -A[(int64_t)r * q + c], Wb[(int64_t)c * s + t]);
            Wb[(int64_t)r * s + t] = acc;
        }
        for (int r = q - 1; r >= 0; --r) {   // U x = y
            cd acc = Wb[(int64_t)r * s + t];
            for (int c = r + 1; c < q; ++c) cfma(acc, -A[(int64_t)r * q + c], Wb[(int64_t)c * s + t]);
            Wb[(int64_t)r * s + t] = cdiv(acc, A[(int64_t)r * q + r]);
        }
    }
}

// z[own point t of leaf B] = sum_b W_B[b][t] v[J_b].  One CTA of 128 threads per
// leaf: the q gathered entries of v are staged in shared memory, then two
// halves of the threads split the sum over b for 64 rows at a time and are
// added in a fixed order.
__global__ void __launch_bounds__(128) k_pc_apply(const int* __restrict__ pc_ptr, const int* __restrict__ pc_idx,
                           const int* __restrict__ own_first, const int* __restrict__ own_cnt,
                           const int64_t* __restrict__ woff, const cd* __restrict__ W, const cd* __restrict__ v,
                           cd* __restrict__ z) {
    extern __shared__ cd vloc[];   // [q] gathered v, then [64] partial sums
    const int B = blockIdx.x;
    const int jb = pc_ptr[B], q = pc_ptr[B + 1] - jb;
    const int s = own_cnt[B];
    const cd* Wb = W + woff[B];
    for (int b = threadIdx.x; b < q; b += blockDim.x) vloc[b] = v[pc_idx[jb + b]];
    cd* part = vloc + q;
    __syncthreads();
    const int half = threadIdx.x >> 6, tl = threadIdx.x & 63;
    const int bh = (q + 1) / 2, b0 = min(q, half * bh), b1 = min(q, b0 + bh);
    for (int t0 = 0; t0 < s; t0 += 64) {
        const int t = t0 + tl;
        cd a[4] = {mk(0, 0), mk(0, 0), mk(0, 0), mk(0, 0)};
        if (t < s) {
            int b = b0;
            for (; b + 8 <= b1; b += 8) {
#pragma unroll
                for (int u = 0; u < 8; ++u) cfma(a[u & 3], Wb[(int64_t)(b + u) * s + t], vloc[b + u]);
            }
            for (; b < b1; ++b) cfma(a[0], Wb[(int64_t)b * s + t], vloc[b]);
        }
        const cd acc = (a[0] + a[1]) + (a[2] + a[3]);
        if (half == 1) part[tl] = acc;
        __syncthreads();
        if (half == 0 && t < s) z[own_first[B] + t] = acc + part[tl];
        __syncthreads();
    }
}

void precond_build(lfmm_geometry_s* g) {
    TreeHost& t = g->tree;
    const int nleaf = g->nleaf;
    std::vector<int> ptr(nleaf + 1, 0), idx, own_pos(nleaf), own_cnt(nleaf), own_first(nleaf), lay(nleaf);
    std::vector<int64_t> aoff(nleaf), woff(nleaf);
    int64_t at = 0, wt = 0;
    for (int li = 0; li < nleaf; ++li) {
        const int B = g->leaf0 + li;
        int q = 0;
        for (int k = t.ufree_ptr[B]; k < t.ufree_ptr[B + 1]; ++k) {
            int S = t.ufree_idx[k];
            if (S == B) own_pos[li] = (int)idx.size() - ptr[li];
            for (int p = t.box_begin[S]; p < t.box_end[S]; ++p) idx.push_back(p);
            q += t.box_end[S] - t.box_begin[S];
        }
        ptr[li + 1] = (int)idx.size();
        own_cnt[li] = t.box_end[B] - t.box_begin[B];
        own_first[li] = t.box_begin[B];
        lay[li] = t.box_layer[B];
        aoff[li] = at;
        at += (int64_t)q * q;
        woff[li] = wt;
        wt += (int64_t)q * own_cnt[li];
    }
    int qmax = 0;
    for (int li = 0; li < nleaf; ++li) qmax = std::max(qmax, ptr[li + 1] - ptr[li]);
    const size_t smem = (size_t)(qmax + 64) * sizeof(cd);
    if (smem > 227 * 1024) throw CudaError{"preconditioner: neighbourhood of " + std::to_string(qmax) +
                                           " points does not fit in shared memory (use a smaller leaf size)"};
    raise_smem_limit((const void*)k_pc_apply, smem, "pc smem");
    g->pc_qmax = qmax;
    g->d_pc_ptr = dupload(g, ptr);
    g->d_pc_idx = dupload(g, idx);
    g->d_pc_woff = dupload(g, woff);
    int* d_own_pos = dupload(g, own_pos);
    int* d_own_cnt = dupload(g, own_cnt);
    int* d_own_first = dupload(g, own_first);
    int* d_lay = dupload(g, lay);
    int64_t* d_aoff = dupload(g, aoff);
    g->d_pc_W = dalloc<cd>(g, (size_t)wt);
    g->pc_w_len = wt;
    cd* Ascr = nullptr;
    int* piv = nullptr;
    cuda_check(cudaMallocAsync((void**)&Ascr, sizeof(cd) * std::max<int64_t>(at, 1), cudaStreamPerThread),
               "malloc pc scratch");
    cuda_check(cudaMallocAsync((void**)&piv, sizeof(int) * std::max<size_t>(idx.size(), 1), cudaStreamPerThread),
               "malloc pc piv");
    k_pc_setup<<<nleaf, 256>>>(g->m, g->d_pc_ptr, g->d_pc_idx, d_own_pos, d_own_cnt, d_aoff, g->d_pc_woff, d_lay,
                               g->d_x, g->d_y, g->d_w, g->d_nx, g->d_ny, Ascr, piv, g->d_pc_W);
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(cudaStreamPerThread);
    dev_release(Ascr);
    dev_release(piv);
    cuda_check(e1, "k_pc_setup");
    cuda_check(e2, "k_pc_setup sync");
    g->pc_own_first = d_own_first;
    g->pc_own_cnt = d_own_cnt;
    g->pc_ready = true;
}

__global__ void k_count_nonfinite(const cd* __restrict__ v, int64_t n, unsigned long long* __restrict__ cnt) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += (isfinite(v[i].x) && isfinite(v[i].y)) ? 0ull : 1ull;
    if (c) atomicAdd(cnt, c);
}

void count_nonfinite(lfmm_geometry_s* g, double out[4]) {
    unsigned long long* d = nullptr;
    cuda_check(cudaMallocAsync((void**)&d, 4 * sizeof(unsigned long long), cudaStreamPerThread), "malloc count");
    cuda_check(cudaMemsetAsync(d, 0, 4 * sizeof(unsigned long long), cudaStreamPerThread), "memset count");
    const cd* bufs[4] = {g->d_nb_val, g->d_m2lf, g->d_m2lr, g->d_pc_W};
    const int64_t lens[4] = {g->nb_nnz, g->m2lf_len, g->m2lr_len, g->pc_ready ? g->pc_w_len : 0};
    for (int i = 0; i < 4; ++i)
        if (bufs[i] && lens[i] > 0)
            k_count_nonfinite<<<152 * 4, 256, 0, cudaStreamPerThread>>>(bufs[i], lens[i], d + i);
    unsigned long long h[4] = {0, 0, 0, 0};
    cuda_check(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, cudaStreamPerThread), "count d2h");
    cuda_check(cudaStreamSynchronize(cudaStreamPerThread), "count sync");
    dev_release(d);
    for (int i = 0; i < 4; ++i) out[i] = (double)h[i];
}

// per reaction table: its non-finite entries (one CTA per key)
__global__ void k_key_nonfinite(const cd* __restrict__ tab, const ReactKey* __restrict__ keys, double* __restrict__ out) {
    const ReactKey K = keys[blockIdx.x];
    const int64_t ne = (int64_t)(2 * K.pT + 1) * (2 * K.pS + 1);
    int c = 0;
    for (int64_t e = threadIdx.x; e < ne; e += blockDim.x) c += (isfinite(tab[K.off + e].x) && isfinite(tab[K.off + e].y)) ? 0 : 1;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    __shared__ int sc[8];
    if ((threadIdx.x & 31) == 0) sc[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sc[i];
        out[blockIdx.x] = (double)t;
    }
}

void react_key_report(lfmm_geometry_s* g, std::vector<double>& out) {
    const int nk = (int)g->rkeys_host.size();
    out.assign((size_t)nk * 8, 0.0);
    if (nk == 0) return;
    double* d = nullptr;
    cuda_check(cudaMallocAsync((void**)&d, sizeof(double) * nk, cudaStreamPerThread), "malloc key report");
    k_key_nonfinite<<<nk, 256, 0, cudaStreamPerThread>>>(g->d_m2lr, g->d_rkeys, d);
    std::vector<double> h(nk);
    cuda_check(cudaMemcpyAsync(h.data(), d, sizeof(double) * nk, cudaMemcpyDeviceToHost, cudaStreamPerThread), "d2h");
    cuda_check(cudaStreamSynchronize(cudaStreamPerThread), "key report");
    dev_release(d);
    for (int k = 0; k < nk; ++k) {
        const ReactKey& K = g->rkeys_host[k];
        const double v[8] = {(double)K.comp, (double)K.level, (double)K.pS, K.X, K.hS, K.hT, K.D, h[k]};
        for (int i = 0; i < 8; ++i) out[(size_t)k * 8 + i] = v[i];
    }
}

void precond_apply_sorted(lfmm_geometry_s* g, const cd* v_sorted, cd* z_sorted, cudaStream_t s) {
    const size_t smem = (size_t)(g->pc_qmax + 64) * sizeof(cd);
    k_pc_apply<<<g->nleaf, 128, smem, s>>>(g->d_pc_ptr, g->d_pc_idx, g->pc_own_first, g->pc_own_cnt, g->d_pc_woff,
                                       g->d_pc_W, v_sorted, z_sorted);
    cuda_check(cudaGetLastError(), "k_pc_apply");
}

}  // namespace lfmm
