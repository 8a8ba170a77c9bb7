// solver.cu -- the full operator, GMRES, the plane-wave right-hand side and the
// scattered field (Secs. 2.2, 3.3, 4.1, 5).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <stdexcept>
#include <vector>

#include "geometry.h"
#include "sommerfeld.cuh"

namespace lfmm {

// ------------------------------------------------------------------ permutations
// caller-order vectors in FP64 (cd) or, with LFMM_C64, single precision (float2):
// widened on the way in, rounded to nearest on the way out
__device__ __forceinline__ cd widen(cd v) { return v; }
__device__ __forceinline__ cd widen(float2 v) { return mk((double)v.x, (double)v.y); }
__device__ __forceinline__ void store_as(cd* p, cd v) { *p = v; }
__device__ __forceinline__ void store_as(float2* p, cd v) { *p = make_float2((float)v.x, (float)v.y); }

template <class T>
__global__ void k_gather(const int* __restrict__ perm, const T* __restrict__ in, cd* __restrict__ out, int64_t n,
                         int nrhs) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * nrhs) return;
    int64_t col = t / n, s = t - col * n;
    out[t] = widen(in[col * n + perm[s]]);
}
template <class T>
__global__ void k_scatter(const int* __restrict__ perm, const cd* __restrict__ in, T* __restrict__ out,
                          int64_t n, int nrhs) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * nrhs) return;
    int64_t col = t / n, s = t - col * n;
    store_as(out + col * n + perm[s], in[t]);
}

template <class T>
static void gather_t(lfmm_geometry_s* g, const T* x_in, cd* x_sorted, int nrhs, cudaStream_t s) {
    int64_t tot = g->n * nrhs;
    k_gather<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g->d_perm, x_in, x_sorted, g->n, nrhs);
    cuda_check(cudaGetLastError(), "k_gather");
    ++g->n_launches;
}
template <class T>
static void scatter_t(lfmm_geometry_s* g, const cd* y_sorted, T* y_out, int nrhs, cudaStream_t s) {
    int64_t tot = g->n * nrhs;
    k_scatter<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(g->d_perm, y_sorted, y_out, g->n, nrhs);
    cuda_check(cudaGetLastError(), "k_scatter");
    ++g->n_launches;
}
void gather_sorted(lfmm_geometry_s* g, const cd* x_in, cd* x_sorted, int nrhs, cudaStream_t s) {
    gather_t(g, x_in, x_sorted, nrhs, s);
}
void scatter_sorted(lfmm_geometry_s* g, const cd* y_sorted, cd* y_out, int nrhs, cudaStream_t s) {
    scatter_t(g, y_sorted, y_out, nrhs, s);
}
void gather_sorted_c64(lfmm_geometry_s* g, const float2* x_in, cd* x_sorted, int nrhs, cudaStream_t s) {
    gather_t(g, x_in, x_sorted, nrhs, s);
}
void scatter_sorted_c64(lfmm_geometry_s* g, const cd* y_sorted, float2* y_out, int nrhs, cudaStream_t s) {
    scatter_t(g, y_sorted, y_out, nrhs, s);
}
__global__ void k_round_c64(const cd* __restrict__ in, float2* __restrict__ out, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) store_as(out + t, in[t]);
}
void round_to_c64(const cd* in, float2* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_round_c64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
    cuda_check(cudaGetLastError(), "k_round_c64");
}

void apply_operator_sorted(lfmm_geometry_s* g, const cd* x_sorted, cd* y_sorted, int nrhs, cudaStream_t s,
                           bool mixed) {
    cuda_check(cudaMemsetAsync(y_sorted, 0, sizeof(cd) * g->n * nrhs, s), "memset y");
    // the stored near field (bound by HBM) on the geometry's side stream, beside the far
    // field (bound by the FP64 pipe); both add into y, the leaf evaluations after it
    cuda_check(cudaEventRecord(g->ev_fork, s), "fork");
    cuda_check(cudaStreamWaitEvent(g->side, g->ev_fork, 0), "fork");
    near_apply(g, x_sorted, y_sorted, nrhs, g->side, mixed);
    cuda_check(cudaEventRecord(g->ev_join, g->side), "join");
    fmm_apply(g, x_sorted, y_sorted, nrhs, s, mixed, g->ev_join);
    cuda_check(cudaStreamWaitEvent(s, g->ev_join, 0), "join");   // also when there is no far field
}

// Several geometries' FP64 operators in shared launches (one launch per stage for all of
// them); each y is what apply_operator_sorted gives for its geometry, bit for bit.  The
// near fields run on the first geometry's side stream beside the far fields.
void apply_operator_batch_sorted(const std::vector<BatchOp>& ops, cudaStream_t s) {
    if (ops.empty()) return;
    for (const BatchOp& op : ops)
        cuda_check(cudaMemsetAsync(op.y, 0, sizeof(cd) * op.g->n * op.nrhs, s), "memset y");
    lfmm_geometry_s* g0 = ops[0].g;
    cuda_check(cudaEventRecord(g0->ev_fork, s), "fork");
    cuda_check(cudaStreamWaitEvent(g0->side, g0->ev_fork, 0), "fork");
    near_apply_batch(ops, g0->side);
    cuda_check(cudaEventRecord(g0->ev_join, g0->side), "join");
    fmm_apply_batch(ops, s, g0->ev_join);
    cuda_check(cudaStreamWaitEvent(s, g0->ev_join, 0), "join");
}

// ------------------------------------------------------------------ BLAS-2 helpers for GMRES
// The Arnoldi step streams the Krylov basis V (n x ncol, column-major, complex128)
// from HBM: h = V^H w reads it once, w -= V h reads it once more.
#define VH_ROWS 512    // rows per block of the V^H w kernel
#define VH_COLS 8      // columns per block (one warp each)

// partial[c * nchunk + chunk] = sum over the chunk's rows of conj(V[c][i]) w[i]
__global__ void __launch_bounds__(256) k_vh_partial(const cd* __restrict__ V, int ncol, int64_t ld,
                                                    const cd* __restrict__ w, int64_t n, cd* __restrict__ partial) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.y * VH_COLS + warp;
    const int64_t r0 = (int64_t)blockIdx.x * VH_ROWS;
    const int64_t r1 = min(r0 + VH_ROWS, n);
    if (c >= ncol) return;   // whole warps only: no block-level synchronisation below
    const cd* v = V + (int64_t)c * ld;
    // 16 rows per lane, four loads of V and w in flight
    cd a0 = mk(0, 0), a1 = mk(0, 0), a2 = mk(0, 0), a3 = mk(0, 0);
    int64_t i = r0 + lane;
    for (; i + 96 < r1; i += 128) {
        cfma(a0, conjc(v[i]), w[i]);
        cfma(a1, conjc(v[i + 32]), w[i + 32]);
        cfma(a2, conjc(v[i + 64]), w[i + 64]);
        cfma(a3, conjc(v[i + 96]), w[i + 96]);
    }
    for (; i < r1; i += 32) cfma(a0, conjc(v[i]), w[i]);
    a0 += a1;
    a2 += a3;
    a0 += a2;
    for (int o = 16; o > 0; o >>= 1) {
        a0.x += __shfl_xor_sync(0xffffffffu, a0.x, o);
        a0.y += __shfl_xor_sync(0xffffffffu, a0.y, o);
    }
    if (lane == 0) partial[(int64_t)c * gridDim.x + blockIdx.x] = a0;
}
// out[c] = sum of the column's partials (one warp per column)
__global__ void k_reduce_partials(const cd* __restrict__ partial, int nchunk, int ncol, cd* __restrict__ out) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= ncol) return;
    cd acc = mk(0, 0);
    for (int i = lane; i < nchunk; i += 32) acc += partial[(int64_t)c * nchunk + i];
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) out[c] = acc;
}
// w -= V h (ncol columns); one thread per row, eight columns per round
__global__ void k_update(const cd* __restrict__ V, int ncol, int64_t ld, const cd* __restrict__ h,
                         cd* __restrict__ w, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cd a[4] = {w[i], mk(0, 0), mk(0, 0), mk(0, 0)};
    int c = 0;
    for (; c + 8 <= ncol; c += 8) {   // eight loads of V in flight
#pragma unroll
        for (int q = 0; q < 8; ++q) cfma(a[q & 3], -V[(int64_t)(c + q) * ld + i], h[c + q]);
    }
    for (; c < ncol; ++c) cfma(a[0], -V[(int64_t)c * ld + i], h[c]);
    w[i] = (a[0] + a[1]) + (a[2] + a[3]);
}
// out = V y  (ncol columns)
__global__ void k_combine(const cd* __restrict__ V, int ncol, int64_t ld, const cd* __restrict__ y,
                          cd* __restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cd a[4] = {mk(0, 0), mk(0, 0), mk(0, 0), mk(0, 0)};
    int c = 0;
    for (; c + 8 <= ncol; c += 8) {
#pragma unroll
        for (int q = 0; q < 8; ++q) cfma(a[q & 3], V[(int64_t)(c + q) * ld + i], y[c + q]);
    }
    for (; c < ncol; ++c) cfma(a[0], V[(int64_t)c * ld + i], y[c]);
    out[i] = (a[0] + a[1]) + (a[2] + a[3]);
}
__global__ void k_scale(const cd* __restrict__ in, double s, cd* __restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = s * in[i];
}
// out = in / sqrt(Re nrm2[0]) (the norm is read on the device; nothing is written if it is 0)
__global__ void k_scale_by_norm(const cd* __restrict__ in, const cd* __restrict__ nrm2, cd* __restrict__ out,
                                int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double h = sqrt(fmax(nrm2[0].x, 0.0));
    if (i < n && h > 0.0) out[i] = (1.0 / h) * in[i];
}
__global__ void k_sub_from(const cd* __restrict__ a, cd* y, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // y = a - y (a residual in place)
    if (i < n) y[i] = a[i] - y[i];
}

struct Blas {
    lfmm_geometry_s* g;
    cudaStream_t s;
    cd* partial;
    cd* dres;     // device results: [0, cap) first pass, [cap, 2 cap) second pass, [2 cap] norm^2
    int cap;
    std::vector<cd> host;
    Blas(lfmm_geometry_s* g_, cudaStream_t s_, int maxcol) : g(g_), s(s_), cap(maxcol + 1) {
        const int64_t nchunk = (g->n + VH_ROWS - 1) / VH_ROWS;
        cuda_check(cudaMallocAsync((void**)&partial, sizeof(cd) * nchunk * cap, s), "malloc partial");
        cuda_check(cudaMallocAsync((void**)&dres, sizeof(cd) * (2 * cap + 1), s), "malloc dres");
        host.resize(2 * cap + 1);
    }
    ~Blas() { cudaFreeAsync(partial, s); cudaFreeAsync(dres, s); }
    // out_dev[0..ncol) = V^H w, on the device, no synchronisation
    void vh(const cd* V, int ncol, int64_t ld, const cd* w, int64_t n, cd* out_dev) {
        const int nchunk = (int)((n + VH_ROWS - 1) / VH_ROWS);
        dim3 grid(nchunk, (ncol + VH_COLS - 1) / VH_COLS);
        k_vh_partial<<<grid, 256, 0, s>>>(V, ncol, ld, w, n, partial);
        k_reduce_partials<<<(ncol + 7) / 8, 256, 0, s>>>(partial, nchunk, ncol, out_dev);
        cuda_check(cudaGetLastError(), "k_vh");
    }
    double norm(const cd* w, int64_t n) {
        vh(w, 1, n, w, n, dres + 2 * cap);
        cuda_check(cudaMemcpyAsync(host.data(), dres + 2 * cap, sizeof(cd), cudaMemcpyDeviceToHost, s), "norm d2h");
        cuda_check(cudaStreamSynchronize(s), "norm sync");
        return std::sqrt(std::max(host[0].x, 0.0));
    }
};

static inline int nblk(int64_t n) { return (int)((n + 255) / 256); }

// One right-hand side; vectors in sorted order on the device.
// mixed_below: the Krylov vectors are multiplied by the FP64 operator while the
// GMRES residual estimate is above this relative value and by the precision form
// once it is below (0: FP64 throughout; > 1: precision form throughout).  This is
// the relaxation of inexact Krylov methods: the operator error a step may carry
// grows as the residual falls, so the first steps get the exact operator.
// The operator of one GMRES solve, always from the fixed vector z into the fixed
// vector w: applied once with plain launches (which also makes every lazy work
// buffer), then captured into a CUDA graph on a private stream and replayed, so
// a Krylov step enqueues one graph instead of the ~25 kernels of a matvec.  A
// geometry with the stage profiler on, or any capture failure, keeps the plain
// launches.
struct OpGraph {
    cudaGraphExec_t exec = nullptr;
    bool tried = false;
    void apply(lfmm_geometry_s* g, const cd* z, cd* w, bool mixed, cudaStream_t s) {
        if (exec) {
            cuda_check(cudaGraphLaunch(exec, s), "graph launch");
            return;
        }
        apply_operator_sorted(g, z, w, 1, s, mixed);
        if (tried || g->prof.on) return;
        tried = true;
        cudaStream_t cs = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); return; }
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            try {
                apply_operator_sorted(g, z, w, 1, cs, mixed);
            } catch (...) {
                ok = false;
            }
            if (cudaStreamEndCapture(cs, &graph) != cudaSuccess) ok = false;
        }
        if (ok && graph && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        cudaGetLastError();   // a failed capture leaves plain launches in use
    }
    ~OpGraph() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

static int gmres_one(lfmm_geometry_s* g, const cd* b, cd* x, double tol, int maxit, bool pre, cudaStream_t s,
                     int* iters, double* res_out, double mixed_below = 0.0, int* mixed_steps = nullptr) {
    const int64_t n = g->n;
    Blas bl(g, s, maxit + 1);
    cd *V = nullptr, *w = nullptr, *z = nullptr, *hd = nullptr;
    // stream-ordered allocations: no device-wide synchronisation, so solves on other
    // streams keep running
    cuda_check(cudaMallocAsync((void**)&V, sizeof(cd) * n * (size_t)(maxit + 1), s), "malloc V");
    cuda_check(cudaMallocAsync((void**)&w, sizeof(cd) * n, s), "malloc w");
    cuda_check(cudaMallocAsync((void**)&z, sizeof(cd) * n, s), "malloc z");
    cuda_check(cudaMallocAsync((void**)&hd, sizeof(cd) * (maxit + 2), s), "malloc h");
    struct Free {
        cd *a, *b, *c, *d;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(a, s); cudaFreeAsync(b, s); cudaFreeAsync(c, s); cudaFreeAsync(d, s); }
    } fr{V, w, z, hd, s};
    double beta = bl.norm(b, n);
    cuda_check(cudaMemsetAsync(x, 0, sizeof(cd) * n, s), "memset x");
    if (beta == 0.0) { *iters = 0; *res_out = 0.0; return 1; }
    OpGraph ops[2];   // the operator z -> w, FP64 and precision form
    k_scale<<<nblk(n), 256, 0, s>>>(b, 1.0 / beta, V, n);
    typedef std::complex<double> C;
    std::vector<std::vector<C>> H;
    std::vector<C> cs, sn, gg(1, C(beta, 0.0));
    int j = 0;
    double res = 1.0;
    for (j = 0; j < maxit; ++j) {
        const cd* vj = V + (int64_t)j * n;
        const bool mixed = res <= mixed_below;
        if (mixed && mixed_steps) ++*mixed_steps;
        if (pre) precond_apply_sorted(g, vj, z, s);
        else cuda_check(cudaMemcpyAsync(z, vj, sizeof(cd) * n, cudaMemcpyDeviceToDevice, s), "z = v_j");
        ops[mixed ? 1 : 0].apply(g, z, w, mixed, s);
        // classical Gram-Schmidt, twice, then the norm; one synchronisation per step
        std::vector<C> h(j + 2, C(0, 0));
        for (int pass = 0; pass < 2; ++pass) {
            cd* hp = bl.dres + pass * bl.cap;
            bl.vh(V, j + 1, n, w, n, hp);
            k_update<<<nblk(n), 256, 0, s>>>(V, j + 1, n, hp, w, n);
        }
        bl.vh(w, 1, n, w, n, bl.dres + 2 * bl.cap);
        k_scale_by_norm<<<nblk(n), 256, 0, s>>>(w, bl.dres + 2 * bl.cap, V + (int64_t)(j + 1) * n, n);
        cuda_check(cudaMemcpyAsync(bl.host.data(), bl.dres, sizeof(cd) * (2 * bl.cap + 1), cudaMemcpyDeviceToHost, s),
                   "arnoldi d2h");
        cuda_check(cudaStreamSynchronize(s), "arnoldi sync");
        for (int c = 0; c <= j; ++c)
            h[c] = C(bl.host[c].x, bl.host[c].y) + C(bl.host[bl.cap + c].x, bl.host[bl.cap + c].y);
        const double hn = std::sqrt(std::max(bl.host[2 * bl.cap].x, 0.0));
        h[j + 1] = C(hn, 0.0);
        // Givens rotations
        for (int i = 0; i < j; ++i) {
            C t = cs[i] * h[i] + sn[i] * h[i + 1];
            h[i + 1] = -std::conj(sn[i]) * h[i] + std::conj(cs[i]) * h[i + 1];
            h[i] = t;
        }
        C a = h[j], c = h[j + 1];
        double r = std::hypot(std::abs(a), std::abs(c));
        C cj, sj;
        if (r == 0) { cj = 1; sj = 0; }
        else if (std::abs(a) == 0) { cj = 0; sj = std::conj(c) / std::abs(c); }
        else { cj = std::abs(a) / r; sj = (a / std::abs(a)) * std::conj(c) / r; }
        h[j] = cj * a + sj * c;
        h[j + 1] = 0;
        cs.push_back(cj); sn.push_back(sj);
        gg.push_back(-std::conj(sj) * gg[j]);
        gg[j] = cj * gg[j];
        H.push_back(h);
        res = std::abs(gg[j + 1]) / beta;
        if (res <= tol || hn == 0.0) { ++j; break; }
    }
    int m = (int)H.size();
    std::vector<C> y(m);
    for (int i = m - 1; i >= 0; --i) {
        C sacc = gg[i];
        for (int k2 = i + 1; k2 < m; ++k2) sacc -= H[k2][i] * y[k2];
        y[i] = sacc / H[i][i];
    }
    std::vector<cd> yh(m);
    for (int i = 0; i < m; ++i) yh[i] = mk(y[i].real(), y[i].imag());
    cuda_check(cudaMemcpyAsync(hd, yh.data(), sizeof(cd) * m, cudaMemcpyHostToDevice, s), "y h2d");
    if (pre) {
        k_combine<<<nblk(n), 256, 0, s>>>(V, m, n, hd, z, n);
        precond_apply_sorted(g, z, x, s);
    } else {
        k_combine<<<nblk(n), 256, 0, s>>>(V, m, n, hd, x, n);
    }
    cuda_check(cudaStreamSynchronize(s), "gmres end");
    *iters = m;
    *res_out = res;
    return res <= tol ? 1 : 0;
}

// Several right-hand sides with the FP64 operator, advanced together: one Krylov
// space per column, and every step multiplies the active columns' preconditioned
// vectors in one block matvec (the block right-hand side of the far field, which
// amortises the translations' loads and launches over the columns).  Each
// column's CGS2 Arnoldi step, Givens rotations and stopping test are those of
// gmres_one and use the same kernels, and a column of a block matvec equals its
// single-column product, so every column's iterates equal a separate solve's.  A
// converged column stops taking steps (its slot in the block is zero).  Returns 1
// if every column reached tol; *last_iters is the last column's step count and
// *worst_res the largest residual estimate.
static int gmres_simul(lfmm_geometry_s* g, const cd* B, cd* X, int nrhs, double tol, int maxit, bool pre,
                       cudaStream_t s, int* last_iters, double* worst_res) {
    const int64_t n = g->n;
    const int64_t ldv = n * (int64_t)(maxit + 1);   // column c's basis at V + c ldv
    const int cap = maxit + 2, per = 2 * cap + 1;   // per column: two CGS passes and the norm
    Blas bl(g, s, maxit + 1);                      // its chunk partials (its results are unused)
    cd *V = nullptr, *Z = nullptr, *W = nullptr, *dres = nullptr, *hd = nullptr;
    cuda_check(cudaMallocAsync((void**)&V, sizeof(cd) * ldv * nrhs, s), "malloc V");
    cuda_check(cudaMallocAsync((void**)&Z, sizeof(cd) * n * nrhs, s), "malloc Z");
    cuda_check(cudaMallocAsync((void**)&W, sizeof(cd) * n * nrhs, s), "malloc W");
    cuda_check(cudaMallocAsync((void**)&dres, sizeof(cd) * per * nrhs, s), "malloc dres");
    cuda_check(cudaMallocAsync((void**)&hd, sizeof(cd) * cap * nrhs, s), "malloc y");
    struct Free {
        cd *a, *b, *c, *d, *e;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(a, s); cudaFreeAsync(b, s); cudaFreeAsync(c, s); cudaFreeAsync(d, s); cudaFreeAsync(e, s); }
    } fr{V, Z, W, dres, hd, s};
    typedef std::complex<double> C;
    std::vector<double> beta(nrhs), res(nrhs, 0.0);
    std::vector<char> active(nrhs, 0);
    std::vector<std::vector<std::vector<C>>> H(nrhs);
    std::vector<std::vector<C>> cs(nrhs), sn(nrhs), gg(nrhs);
    cuda_check(cudaMemsetAsync(X, 0, sizeof(cd) * n * nrhs, s), "memset x");
    for (int c = 0; c < nrhs; ++c) {
        beta[c] = bl.norm(B + (int64_t)c * n, n);
        gg[c].assign(1, C(beta[c], 0.0));
        if (beta[c] > 0.0) {
            active[c] = 1;
            res[c] = 1.0;
            k_scale<<<nblk(n), 256, 0, s>>>(B + (int64_t)c * n, 1.0 / beta[c], V + (int64_t)c * ldv, n);
        }
    }
    std::vector<cd> hres((size_t)per * nrhs);
    for (int j = 0; j < maxit; ++j) {
        bool any = false;
        for (int c = 0; c < nrhs; ++c) any |= active[c] != 0;
        if (!any) break;
        for (int c = 0; c < nrhs; ++c) {
            cd* zc = Z + (int64_t)c * n;
            const cd* vj = V + (int64_t)c * ldv + (int64_t)j * n;
            if (!active[c]) cuda_check(cudaMemsetAsync(zc, 0, sizeof(cd) * n, s), "z = 0");
            else if (pre) precond_apply_sorted(g, vj, zc, s);
            else cuda_check(cudaMemcpyAsync(zc, vj, sizeof(cd) * n, cudaMemcpyDeviceToDevice, s), "z = v_j");
        }
        apply_operator_sorted(g, Z, W, nrhs, s, false);
        for (int c = 0; c < nrhs; ++c) {
            if (!active[c]) continue;
            cd* wc = W + (int64_t)c * n;
            const cd* Vc = V + (int64_t)c * ldv;
            cd* base = dres + (int64_t)c * per;
            for (int pass = 0; pass < 2; ++pass) {
                bl.vh(Vc, j + 1, n, wc, n, base + pass * cap);
                k_update<<<nblk(n), 256, 0, s>>>(Vc, j + 1, n, base + pass * cap, wc, n);
            }
            bl.vh(wc, 1, n, wc, n, base + 2 * cap);
            k_scale_by_norm<<<nblk(n), 256, 0, s>>>(wc, base + 2 * cap, V + (int64_t)c * ldv + (int64_t)(j + 1) * n, n);
        }
        cuda_check(cudaMemcpyAsync(hres.data(), dres, sizeof(cd) * per * nrhs, cudaMemcpyDeviceToHost, s), "arnoldi d2h");
        cuda_check(cudaStreamSynchronize(s), "arnoldi sync");
        for (int c = 0; c < nrhs; ++c) {
            if (!active[c]) continue;
            const cd* hr = hres.data() + (size_t)c * per;
            std::vector<C> h(j + 2, C(0, 0));
            for (int q = 0; q <= j; ++q) h[q] = C(hr[q].x, hr[q].y) + C(hr[cap + q].x, hr[cap + q].y);
            const double hn = std::sqrt(std::max(hr[2 * cap].x, 0.0));
            h[j + 1] = C(hn, 0.0);
            for (int i = 0; i < j; ++i) {
                C t = cs[c][i] * h[i] + sn[c][i] * h[i + 1];
                h[i + 1] = -std::conj(sn[c][i]) * h[i] + std::conj(cs[c][i]) * h[i + 1];
                h[i] = t;
            }
            C a = h[j], e = h[j + 1];
            double r = std::hypot(std::abs(a), std::abs(e));
            C cj, sj;
            if (r == 0) { cj = 1; sj = 0; }
            else if (std::abs(a) == 0) { cj = 0; sj = std::conj(e) / std::abs(e); }
            else { cj = std::abs(a) / r; sj = (a / std::abs(a)) * std::conj(e) / r; }
            h[j] = cj * a + sj * e;
            h[j + 1] = 0;
            cs[c].push_back(cj); sn[c].push_back(sj);
            gg[c].push_back(-std::conj(sj) * gg[c][j]);
            gg[c][j] = cj * gg[c][j];
            H[c].push_back(h);
            res[c] = std::abs(gg[c][j + 1]) / beta[c];
            if (res[c] <= tol || hn == 0.0) active[c] = 0;
        }
    }
    int all = 1;
    double worst = 0.0;
    for (int c = 0; c < nrhs; ++c) {
        worst = std::max(worst, res[c]);
        if (beta[c] == 0.0) continue;
        all &= res[c] <= tol ? 1 : 0;
        const int m = (int)H[c].size();
        std::vector<C> y(m);
        for (int i = m - 1; i >= 0; --i) {
            C sacc = gg[c][i];
            for (int k2 = i + 1; k2 < m; ++k2) sacc -= H[c][k2][i] * y[k2];
            y[i] = sacc / H[c][i][i];
        }
        std::vector<cd> yh(m);
        for (int i = 0; i < m; ++i) yh[i] = mk(y[i].real(), y[i].imag());
        cd* yd = hd + (int64_t)c * cap;
        cuda_check(cudaMemcpyAsync(yd, yh.data(), sizeof(cd) * m, cudaMemcpyHostToDevice, s), "y h2d");
        cuda_check(cudaStreamSynchronize(s), "y h2d");   // yh is a local host buffer
        const cd* Vc = V + (int64_t)c * ldv;
        cd* xc = X + (int64_t)c * n;
        if (pre) {
            cd* zc = Z + (int64_t)c * n;
            k_combine<<<nblk(n), 256, 0, s>>>(Vc, m, n, yd, zc, n);
            precond_apply_sorted(g, zc, xc, s);
        } else {
            k_combine<<<nblk(n), 256, 0, s>>>(Vc, m, n, yd, xc, n);
        }
    }
    cuda_check(cudaStreamSynchronize(s), "gmres end");
    *last_iters = (int)H[nrhs - 1].size();
    *worst_res = worst;
    return all;
}

__global__ void k_add(cd* __restrict__ x, const cd* __restrict__ d, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = x[i] + d[i];
}

// GMRES for every column.  precision 0: the FP64 operator throughout.
// precision 1: relaxed mixed precision.  The relative difference eps of the two
// operators is measured on b; GMRES runs to 0.3 tol with FP64 products until its
// residual estimate falls below 0.03 tol / eps and with the precision form after
// that, in one Krylov space.  The FP64 residual b - A x is then recomputed; while it
// is above tol, refinement steps solve A d = r the same way (at most 4, stopping
// when a step no longer halves ||r||).
// restart m > 0: GMRES(m).  A pass (the first solve, a restart cycle or a refinement
// step) builds at most m Krylov vectors for the correction d of A d = r, with
// r = b - A x recomputed with the FP64 operator before each pass, and passes repeat
// until that residual reaches tol or max_iter steps have been taken in all.  With the
// precision form, a pass that ends at m steps is a restart, not a stall.
int gmres_sorted(lfmm_geometry_s* g, const cd* b, cd* x, int nrhs, double tol, int maxit, bool pre,
                 cudaStream_t s, lfmm_gmres_info* info, int precision, int restart) {
    auto t0 = std::chrono::steady_clock::now();
    const int64_t n = g->n;
    int all = 1, it = 0, outer_last = 0, f64_last = 0;
    double worst = 0.0, worst_true = 0.0, worst_opdiff = 0.0;
    cd *r = nullptr, *d = nullptr, *y2 = nullptr;
    cuda_check(cudaMallocAsync((void**)&r, sizeof(cd) * n, s), "malloc r");
    cuda_check(cudaMallocAsync((void**)&d, sizeof(cd) * n, s), "malloc d");
    cuda_check(cudaMallocAsync((void**)&y2, sizeof(cd) * n, s), "malloc y2");
    struct Free {
        cd *a, *b, *c;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(a, s); cudaFreeAsync(b, s); cudaFreeAsync(c, s); }
    } fr{r, d, y2, s};
    Blas bl(g, s, 2);
    if (precision == 0 && nrhs > 1 && restart == 0) {
        // all columns at once when their Krylov bases fit in a quarter of the free memory
        size_t free_b = 0, total_b = 0;
        cuda_check(cudaMemGetInfo(&free_b, &total_b), "memory info");
        const double need = 16.0 * (double)n * (double)(maxit + 1) * nrhs + 48.0 * (double)n * nrhs;
        if (need <= 0.25 * (double)free_b) {
            double est = 0.0;
            int ok = gmres_simul(g, b, x, nrhs, tol, maxit, pre, s, &it, &est);
            // true residuals: one block product
            cd* R = nullptr;
            cuda_check(cudaMallocAsync((void**)&R, sizeof(cd) * n * nrhs, s), "malloc R");
            apply_operator_sorted(g, x, R, nrhs, s);
            for (int c = 0; c < nrhs; ++c) {
                const cd* bc = b + (int64_t)c * n;
                cd* rc = R + (int64_t)c * n;
                k_sub_from<<<nblk(n), 256, 0, s>>>(bc, rc, n);
                const double bn = bl.norm(bc, n), rn = bl.norm(rc, n);
                worst_true = std::max(worst_true, bn > 0.0 ? rn / bn : 0.0);
            }
            cudaFreeAsync(R, s);
            if (info) {
                info->iterations = it;
                info->converged = ok;
                info->rel_residual = est;
                info->true_rel_residual = worst_true;
                info->solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                info->refinements = 0;
                info->fp64_matvecs = 1;
                info->op_rel_diff = 0.0;
            }
            return ok;
        }
    }
    // ||(A_mixed - A) v|| / ||A v||
    auto op_diff = [&](const cd* v) {
        apply_operator_sorted(g, v, y2, 1, s, true);
        apply_operator_sorted(g, v, d, 1, s);
        const double an = bl.norm(d, n);
        k_sub_from<<<nblk(n), 256, 0, s>>>(y2, d, n);
        const double dn = bl.norm(d, n);
        return an > 0.0 ? dn / an : 0.0;
    };
    for (int c = 0; c < nrhs; ++c) {
        const cd* bc = b + (int64_t)c * n;
        cd* xc = x + (int64_t)c * n;
        double res = 0.0, rn = 0.0;
        const double bn = bl.norm(bc, n);
        int ok = 0, outer = 0, f64 = 0;
        if (precision == 0 && restart == 0) {
            ok = gmres_one(g, bc, xc, tol, maxit, pre, s, &it, &res);
            apply_operator_sorted(g, xc, r, 1, s);
            k_sub_from<<<nblk(n), 256, 0, s>>>(bc, r, n);
            rn = bl.norm(r, n);
            f64 = 1;
            // the estimate reached tol but the recomputed residual did not (rounding drift over a
            // long Krylov run): refinement passes A d = r, x += d, while steps remain and each
            // pass at least halves ||r||
            while (bn > 0.0 && rn > tol * bn && it < maxit && outer < 4) {
                int its = 0;
                double rr = 0.0;
                gmres_one(g, r, d, std::min(0.5, 0.5 * tol * bn / rn), maxit - it, pre, s, &its, &rr);
                it += its;
                k_add<<<nblk(n), 256, 0, s>>>(xc, d, n);
                apply_operator_sorted(g, xc, r, 1, s);
                k_sub_from<<<nblk(n), 256, 0, s>>>(bc, r, n);
                ++f64;
                ++outer;
                const double rn_new = bl.norm(r, n);
                const bool stalled = rn_new > 0.5 * rn;
                rn = rn_new;
                if (stalled) break;
            }
            if (outer > 0) {
                ok = rn <= tol * bn ? 1 : 0;
                res = bn > 0.0 ? rn / bn : 0.0;
            }
        } else if (precision == 0) {
            // GMRES(m): each cycle solves A d = r from a fresh Krylov space of at most m vectors
            cuda_check(cudaMemsetAsync(xc, 0, sizeof(cd) * n, s), "memset x");
            cuda_check(cudaMemcpyAsync(r, bc, sizeof(cd) * n, cudaMemcpyDeviceToDevice, s), "r = b");
            rn = bn;
            int total = 0;
            while (bn > 0.0 && rn > tol * bn && total < maxit) {
                const double tol_in = (outer == 0) ? tol : tol * bn / rn;
                int its = 0;
                double rr = 0.0;
                gmres_one(g, r, d, tol_in, std::min(restart, maxit - total), pre, s, &its, &rr);
                total += its;
                f64 += its;
                k_add<<<nblk(n), 256, 0, s>>>(xc, d, n);
                apply_operator_sorted(g, xc, r, 1, s);
                k_sub_from<<<nblk(n), 256, 0, s>>>(bc, r, n);
                ++f64;
                ++outer;
                rn = bl.norm(r, n);
            }
            it = total;
            ok = (bn == 0.0 || rn <= tol * bn) ? 1 : 0;
            res = bn > 0.0 ? rn / bn : 0.0;
        } else {
            const double eps = (bn > 0.0) ? std::max(op_diff(bc), 1e-300) : 1e-300;
            f64 += 1;
            // the first pass aims below tol so that the gap between its residual estimate
            // and the FP64 residual (left by the mixed products) rarely needs a second pass
            const double tol1 = 0.3 * tol;
            const double below = 0.1 * tol1 / eps;
            cuda_check(cudaMemsetAsync(xc, 0, sizeof(cd) * n, s), "memset x");
            cuda_check(cudaMemcpyAsync(r, bc, sizeof(cd) * n, cudaMemcpyDeviceToDevice, s), "r = b");
            rn = bn;
            int total = 0;
            while (bn > 0.0 && rn > tol * bn && total < maxit && (restart > 0 || outer < 5)) {
                const double tol_in = (outer == 0) ? tol1 : std::min(0.5, 0.5 * tol * bn / rn);
                const double below_in = (outer == 0) ? below : below * bn / rn;
                const int cap = restart > 0 ? std::min(restart, maxit - total) : maxit - total;
                int its = 0, msteps = 0;
                double rr = 0.0;
                const int reached = gmres_one(g, r, d, tol_in, cap, pre, s, &its, &rr, below_in, &msteps);
                total += its;
                f64 += its - msteps;
                k_add<<<nblk(n), 256, 0, s>>>(xc, d, n);
                apply_operator_sorted(g, xc, r, 1, s);
                k_sub_from<<<nblk(n), 256, 0, s>>>(bc, r, n);
                ++f64;
                ++outer;
                const double rn_new = bl.norm(r, n);
                const bool stalled = rn_new > 0.5 * rn && (restart == 0 || reached);
                rn = rn_new;
                if (stalled) break;
            }
            it = total;
            ok = (bn == 0.0 || rn <= tol * bn) ? 1 : 0;
            res = bn > 0.0 ? rn / bn : 0.0;
            worst_opdiff = std::max(worst_opdiff, eps < 1e-299 ? 0.0 : eps);
        }
        all &= ok;
        worst = std::max(worst, res);
        worst_true = std::max(worst_true, bn > 0 ? rn / bn : 0.0);
        outer_last = outer;
        f64_last = f64;
    }
    if (info) {
        info->iterations = it;
        info->converged = all;
        info->rel_residual = worst;
        info->true_rel_residual = worst_true;
        info->solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->refinements = outer_last;
        info->fp64_matvecs = f64_last;
        info->op_rel_diff = worst_opdiff;
    }
    return all;
}

// ------------------------------------------------------------------ lockstep solves (serving)
// The serving loop's batched form: several solves, each of its own geometry with one
// right-hand side, advanced together, one Krylov step of each per round.  The FP64
// products of a round share launches (apply_operator_batch_sorted: one launch per stage
// for all of them); precision-form products stay per geometry.  A solve's passes, Arnoldi
// steps (CGS2), Givens rotations, stopping tests and refinement are those of gmres_sorted
// with restart 0 and one column (gmres_one), with the same kernels in the same order, and
// a shared launch gives each geometry the bits of its own launches, so a solve's result
// equals the same solve alone, bit for bit.  A round runs on one stream with one host
// synchronisation for all of its solves.
struct BatchSolve {
    typedef std::complex<double> C;
    lfmm_geometry_s* g = nullptr;
    int64_t n = 0;
    double tol = 1e-8;
    int maxit = 1000, precision = 0;
    bool pre = true;
    cd *b = nullptr, *x = nullptr;   // sorted order, owned
    // the driver (gmres_sorted)
    bool done = false;
    int ok = 0, outer = 0, total = 0, f64 = 0, it = 0;
    double bn = 0, rn = 0, eps = 0, below = 0, res_est = 0;
    cd *r = nullptr, *d = nullptr, *y2 = nullptr;
    // the current pass (gmres_one)
    bool in_pass = false;
    const cd* prhs = nullptr;
    cd* pout = nullptr;
    double beta = 0, res = 1, tol_in = 0, below_in = 0;
    int cap = 0, msteps = 0;
    bool mixed_step = false;
    cd *V = nullptr, *w = nullptr, *z = nullptr, *hd = nullptr;
    Blas* bl = nullptr;      // Arnoldi results (columns up to maxit + 1)
    Blas* bo = nullptr;      // norms of the driver
    cd* hpin = nullptr;      // pinned copy of bl->dres
    std::vector<std::vector<C>> H;
    std::vector<C> cs, sn, gg;
    OpGraph opm;             // the precision-form operator z -> w
    std::chrono::steady_clock::time_point t0;
    cudaStream_t st = nullptr;   // the solve's own stream: everything but the shared products
    cudaEvent_t ev = nullptr;    // its direction z is ready
};

BatchSolve* batch_solve_create(lfmm_geometry_s* g, const cd* b_in, double tol, int maxit, bool pre, int precision,
                               cudaStream_t s) {
    BatchSolve* S = new BatchSolve();
    S->g = g;
    S->n = g->n;
    S->tol = tol;
    S->maxit = maxit;
    S->pre = pre;
    S->precision = precision;
    if (pre && !g->pc_ready) precond_build(g);
    const int64_t n = g->n;
    cuda_check(cudaMallocAsync((void**)&S->b, sizeof(cd) * n, s), "malloc b");
    cuda_check(cudaMallocAsync((void**)&S->x, sizeof(cd) * n, s), "malloc x");
    gather_sorted(g, b_in, S->b, 1, s);
    cuda_check(cudaStreamSynchronize(s), "batch solve create");
    return S;
}

static void bs_pass_start(BatchSolve& S, const cd* rhs, cd* out, double tol_in, double below_in, int cap,
                          cudaStream_t s) {
    const int64_t n = S.n;
    if (!S.V) {   // the largest pass: maxit steps
        cuda_check(cudaMallocAsync((void**)&S.V, sizeof(cd) * n * (size_t)(S.maxit + 1), s), "malloc V");
        cuda_check(cudaMallocAsync((void**)&S.w, sizeof(cd) * n, s), "malloc w");
        cuda_check(cudaMallocAsync((void**)&S.z, sizeof(cd) * n, s), "malloc z");
        cuda_check(cudaMallocAsync((void**)&S.hd, sizeof(cd) * (S.maxit + 2), s), "malloc h");
        S.bl = new Blas(S.g, s, S.maxit + 1);
        cuda_check(cudaMallocHost((void**)&S.hpin, sizeof(cd) * (2 * S.bl->cap + 1)), "pinned h");
    }
    S.prhs = rhs;
    S.pout = out;
    S.tol_in = tol_in;
    S.below_in = below_in;
    S.cap = cap;
    S.msteps = 0;
    S.beta = S.bl->norm(rhs, n);
    cuda_check(cudaMemsetAsync(out, 0, sizeof(cd) * n, s), "memset x");
    S.H.clear(); S.cs.clear(); S.sn.clear();
    S.gg.assign(1, BatchSolve::C(S.beta, 0.0));
    S.res = 1.0;
    S.in_pass = S.beta != 0.0;
    if (!S.in_pass) S.res = 0.0;
    else k_scale<<<nblk(n), 256, 0, s>>>(rhs, 1.0 / S.beta, S.V, n);
}

// ||(A_mixed - A) v|| / ||A v||, as gmres_sorted measures it
static double bs_op_diff(BatchSolve& S, const cd* v, cudaStream_t s) {
    apply_operator_sorted(S.g, v, S.y2, 1, s, true);
    apply_operator_sorted(S.g, v, S.d, 1, s);
    const double an = S.bo->norm(S.d, S.n);
    k_sub_from<<<nblk(S.n), 256, 0, s>>>(S.y2, S.d, S.n);
    const double dn = S.bo->norm(S.d, S.n);
    return an > 0.0 ? dn / an : 0.0;
}

// the next pass of the refinement loop of gmres_sorted (precision 1), or the end
static void bs_next_or_finish(BatchSolve& S, cudaStream_t s) {
    const double tol1 = 0.3 * S.tol;
    if (S.bn > 0.0 && S.rn > S.tol * S.bn && S.total < S.maxit && S.outer < 5) {
        const double tol_in = (S.outer == 0) ? tol1 : std::min(0.5, 0.5 * S.tol * S.bn / S.rn);
        const double below_in = (S.outer == 0) ? S.below : S.below * S.bn / S.rn;
        bs_pass_start(S, S.r, S.d, tol_in, below_in, S.maxit - S.total, s);
        if (S.in_pass) return;
        // a zero residual: the pass is empty (as gmres_one with beta = 0)
    }
    if (!S.in_pass) {
        S.it = S.total;
        S.ok = (S.bn == 0.0 || S.rn <= S.tol * S.bn) ? 1 : 0;
        S.res_est = S.bn > 0.0 ? S.rn / S.bn : 0.0;
        S.done = true;
    }
}

void batch_solve_begin(BatchSolve* Sp, cudaStream_t engine) {
    BatchSolve& S = *Sp;
    S.t0 = std::chrono::steady_clock::now();
    cuda_check(cudaStreamCreateWithFlags(&S.st, cudaStreamNonBlocking), "solve stream");
    cuda_check(cudaEventCreateWithFlags(&S.ev, cudaEventDisableTiming), "solve event");
    cuda_check(cudaEventRecord(S.ev, engine), "event");      // after the set-up seen by the engine
    cuda_check(cudaStreamWaitEvent(S.st, S.ev, 0), "wait");
    cudaStream_t s = S.st;
    const int64_t n = S.n;
    cuda_check(cudaMallocAsync((void**)&S.r, sizeof(cd) * n, s), "malloc r");
    cuda_check(cudaMallocAsync((void**)&S.d, sizeof(cd) * n, s), "malloc d");
    cuda_check(cudaMallocAsync((void**)&S.y2, sizeof(cd) * n, s), "malloc y2");
    S.bo = new Blas(S.g, s, 2);
    S.bn = S.bo->norm(S.b, n);
    if (S.precision == 0) {
        bs_pass_start(S, S.b, S.x, S.tol, 0.0, S.maxit, s);
        if (!S.in_pass) {   // b = 0
            S.it = 0; S.res_est = 0.0; S.ok = 1;
            apply_operator_sorted(S.g, S.x, S.r, 1, s);
            k_sub_from<<<nblk(n), 256, 0, s>>>(S.b, S.r, n);
            S.rn = S.bo->norm(S.r, n);
            S.f64 = 1;
            S.done = true;
        }
        return;
    }
    S.eps = (S.bn > 0.0) ? std::max(bs_op_diff(S, S.b, s), 1e-300) : 1e-300;
    S.f64 += 1;
    S.below = 0.1 * (0.3 * S.tol) / S.eps;
    cuda_check(cudaMemsetAsync(S.x, 0, sizeof(cd) * n, s), "memset x");
    cuda_check(cudaMemcpyAsync(S.r, S.b, sizeof(cd) * n, cudaMemcpyDeviceToDevice, s), "r = b");
    S.rn = S.bn;
    bs_next_or_finish(S, s);
}

// end of a pass: the iterate from the Krylov basis (gmres_one's end), then the driver
static void bs_pass_end(BatchSolve& S, cudaStream_t s) {
    typedef BatchSolve::C C;
    const int64_t n = S.n;
    const int m = (int)S.H.size();
    std::vector<C> y(m);
    for (int i = m - 1; i >= 0; --i) {
        C sacc = S.gg[i];
        for (int k2 = i + 1; k2 < m; ++k2) sacc -= S.H[k2][i] * y[k2];
        y[i] = sacc / S.H[i][i];
    }
    std::vector<cd> yh(m);
    for (int i = 0; i < m; ++i) yh[i] = mk(y[i].real(), y[i].imag());
    cuda_check(cudaMemcpyAsync(S.hd, yh.data(), sizeof(cd) * m, cudaMemcpyHostToDevice, s), "y h2d");
    if (S.pre) {
        k_combine<<<nblk(n), 256, 0, s>>>(S.V, m, n, S.hd, S.z, n);
        precond_apply_sorted(S.g, S.z, S.pout, s);
    } else {
        k_combine<<<nblk(n), 256, 0, s>>>(S.V, m, n, S.hd, S.pout, n);
    }
    cuda_check(cudaStreamSynchronize(s), "pass end");   // yh is a local host buffer
    S.in_pass = false;
    const int its = m;
    if (S.precision == 0) {
        if (S.outer == 0) {   // the first pass solved for x itself
            S.it = its;
            S.res_est = S.res;
            S.ok = S.res <= S.tol ? 1 : 0;
            S.f64 = 1;
        } else {              // a refinement pass: x += d
            S.it += its;
            k_add<<<nblk(n), 256, 0, s>>>(S.x, S.d, n);
            ++S.f64;
        }
        apply_operator_sorted(S.g, S.x, S.r, 1, s);
        k_sub_from<<<nblk(n), 256, 0, s>>>(S.b, S.r, n);
        const double rn_new = S.bo->norm(S.r, n);
        const bool stalled = S.outer > 0 && rn_new > 0.5 * S.rn;
        S.rn = rn_new;
        if (S.outer > 0) {
            S.ok = S.rn <= S.tol * S.bn ? 1 : 0;
            S.res_est = S.bn > 0.0 ? S.rn / S.bn : 0.0;
        }
        // as gmres_sorted: refinement while the recomputed residual misses tol
        if (!stalled && S.bn > 0.0 && S.rn > S.tol * S.bn && S.it < S.maxit && S.outer < 4) {
            ++S.outer;
            bs_pass_start(S, S.r, S.d, std::min(0.5, 0.5 * S.tol * S.bn / S.rn), 0.0, S.maxit - S.it, s);
            if (S.in_pass) return;
            --S.outer;
        }
        S.done = true;
        return;
    }
    S.total += its;
    S.f64 += its - S.msteps;
    k_add<<<nblk(n), 256, 0, s>>>(S.x, S.d, n);
    apply_operator_sorted(S.g, S.x, S.r, 1, s);
    k_sub_from<<<nblk(n), 256, 0, s>>>(S.b, S.r, n);
    ++S.f64;
    ++S.outer;
    const double rn_new = S.bo->norm(S.r, n);
    const bool stalled = rn_new > 0.5 * S.rn;
    S.rn = rn_new;
    if (stalled) {
        S.it = S.total;
        S.ok = (S.bn == 0.0 || S.rn <= S.tol * S.bn) ? 1 : 0;
        S.res_est = S.bn > 0.0 ? S.rn / S.bn : 0.0;
        S.done = true;
        return;
    }
    bs_next_or_finish(S, s);
}

void batch_solve_round(const std::vector<BatchSolve*>& all, cudaStream_t s) {
    typedef BatchSolve::C C;
    std::vector<BatchSolve*> act;
    for (BatchSolve* S : all)
        if (!S->done && S->in_pass) act.push_back(S);
    if (act.empty()) return;
    // preconditioned directions, each on its solve's stream; precision-form products there too
    std::vector<BatchOp> ops;
    for (BatchSolve* S : act) {
        const int j = (int)S->H.size();
        const cd* vj = S->V + (int64_t)j * S->n;
        S->mixed_step = S->res <= S->below_in;
        if (S->mixed_step) ++S->msteps;
        if (S->pre) precond_apply_sorted(S->g, vj, S->z, S->st);
        else cuda_check(cudaMemcpyAsync(S->z, vj, sizeof(cd) * S->n, cudaMemcpyDeviceToDevice, S->st), "z = v_j");
        if (S->mixed_step) {
            S->opm.apply(S->g, S->z, S->w, true, S->st);
        } else {
            cuda_check(cudaEventRecord(S->ev, S->st), "event");
            cuda_check(cudaStreamWaitEvent(s, S->ev, 0), "wait for z");
            ops.push_back(BatchOp{S->g, S->z, S->w, 1});
        }
    }
    // the FP64 products in shared launches on the engine's stream
    if (!ops.empty()) {
        apply_operator_batch_sorted(ops, s);
        cudaEvent_t done = nullptr;
        cuda_check(cudaEventCreateWithFlags(&done, cudaEventDisableTiming), "event");
        cuda_check(cudaEventRecord(done, s), "event");
        for (BatchSolve* S : act)
            if (!S->mixed_step) cuda_check(cudaStreamWaitEvent(S->st, done, 0), "wait for the products");
        cudaEventDestroy(done);   // released once the waits above have been satisfied
    }
    // Arnoldi steps on each solve's stream, then one wait for all of them
    for (BatchSolve* S : act) {
        const int j = (int)S->H.size();
        const int64_t n = S->n;
        Blas& bl = *S->bl;
        for (int pass = 0; pass < 2; ++pass) {
            cd* hp = bl.dres + pass * bl.cap;
            bl.vh(S->V, j + 1, n, S->w, n, hp);
            k_update<<<nblk(n), 256, 0, S->st>>>(S->V, j + 1, n, hp, S->w, n);
        }
        bl.vh(S->w, 1, n, S->w, n, bl.dres + 2 * bl.cap);
        k_scale_by_norm<<<nblk(n), 256, 0, S->st>>>(S->w, bl.dres + 2 * bl.cap, S->V + (int64_t)(j + 1) * n, n);
        cuda_check(cudaMemcpyAsync(S->hpin, bl.dres, sizeof(cd) * (2 * bl.cap + 1), cudaMemcpyDeviceToHost, S->st),
                   "arnoldi d2h");
    }
    for (BatchSolve* S : act) cuda_check(cudaStreamSynchronize(S->st), "round sync");
    for (BatchSolve* S : act) {
        const int j = (int)S->H.size();
        const int capb = S->bl->cap;
        const cd* hh = S->hpin;
        std::vector<C> h(j + 2, C(0, 0));
        for (int c = 0; c <= j; ++c) h[c] = C(hh[c].x, hh[c].y) + C(hh[capb + c].x, hh[capb + c].y);
        const double hn = std::sqrt(std::max(hh[2 * capb].x, 0.0));
        h[j + 1] = C(hn, 0.0);
        for (int i = 0; i < j; ++i) {
            C t = S->cs[i] * h[i] + S->sn[i] * h[i + 1];
            h[i + 1] = -std::conj(S->sn[i]) * h[i] + std::conj(S->cs[i]) * h[i + 1];
            h[i] = t;
        }
        C a = h[j], c = h[j + 1];
        double rr = std::hypot(std::abs(a), std::abs(c));
        C cj, sj;
        if (rr == 0) { cj = 1; sj = 0; }
        else if (std::abs(a) == 0) { cj = 0; sj = std::conj(c) / std::abs(c); }
        else { cj = std::abs(a) / rr; sj = (a / std::abs(a)) * std::conj(c) / rr; }
        h[j] = cj * a + sj * c;
        h[j + 1] = 0;
        S->cs.push_back(cj); S->sn.push_back(sj);
        S->gg.push_back(-std::conj(sj) * S->gg[j]);
        S->gg[j] = cj * S->gg[j];
        S->H.push_back(h);
        S->res = std::abs(S->gg[j + 1]) / S->beta;
        if (S->res <= S->tol_in || hn == 0.0 || (int)S->H.size() >= S->cap) bs_pass_end(*S, S->st);
    }
}

bool batch_solve_done(const BatchSolve* S) { return S->done; }

void batch_solve_finish(BatchSolve* S, cd* x_out, lfmm_gmres_info* info, cudaStream_t s) {
    if (S->st) cuda_check(cudaStreamSynchronize(S->st), "solve stream");
    scatter_sorted(S->g, S->x, x_out, 1, s);
    if (info) {
        info->iterations = S->it;
        info->converged = S->ok;
        info->rel_residual = S->res_est;
        info->true_rel_residual = S->bn > 0 ? S->rn / S->bn : 0.0;
        info->solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - S->t0).count();
        info->refinements = S->outer;
        info->fp64_matvecs = S->f64;
        info->op_rel_diff = (S->precision == 1 && S->eps >= 1e-299) ? S->eps : 0.0;
    }
    cuda_check(cudaStreamSynchronize(s), "batch solve finish");
}

void batch_solve_destroy(BatchSolve* S, cudaStream_t s) {
    if (!S) return;
    if (S->st) cudaStreamSynchronize(S->st);
    for (cd* p : {S->b, S->x, S->r, S->d, S->y2, S->V, S->w, S->z, S->hd})
        if (p) cudaFreeAsync(p, s);
    delete S->bl;   // frees on the solve's stream
    delete S->bo;
    if (S->st) cudaStreamSynchronize(S->st);
    cudaStreamSynchronize(s);
    if (S->hpin) cudaFreeHost(S->hpin);
    if (S->ev) cudaEventDestroy(S->ev);
    if (S->st) cudaStreamDestroy(S->st);
    delete S;
}

// ------------------------------------------------------------------ right-hand side (Sec. 2.2)
// Background field of a plane wave, by the generalized reflection/transmission
// recursions of the paper (A_l, B_l after eq. TLhelmholtztotallayer2) written
// with each layer's waves referenced at its own interfaces.
__global__ void k_rhs(MediumDev m, const double* __restrict__ px, const double* __restrict__ py,
                      const int* __restrict__ layer, const double* __restrict__ angles, int nrhs, int64_t n,
                      cd* __restrict__ b) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * nrhs) return;
    const int col = (int)(t / n);
    const int64_t i = t - (int64_t)col * n;
    const int L = m.nl - 1;
    const double th = angles[col];
    const double kx = m.k[0] * cos(th);
    const int l = layer[i];
    const double x = px[i], y = py[i];
    cd lam = mk(kx, 0.0);
    cd kyv[LFMM_MAXLAY], e[LFMM_MAXLAY], Rl[LFMM_MAXLAY], Rd[LFMM_MAXLAY];
    for (int q = 0; q <= L; ++q) {
        kyv[q] = ky_of(m.k[q], lam);
        e[q] = (q >= 1 && q <= L - 1) ? eikh(kyv[q], m.yint[q - 1] - m.yint[q]) : mk(0.0, 0.0);
    }
    for (int q = 0; q < L; ++q) {
        cd A = m.eta[q] * kyv[q], B = m.eta[q + 1] * kyv[q + 1];
        Rl[q] = cdiv(A - B, A + B);
    }
    for (int q = 0; q <= L; ++q) Rd[q] = mk(0.0, 0.0);
    for (int q = L - 1; q >= 0; --q) {
        if (q == L - 1) Rd[q] = Rl[q];
        else {
            cd tt = Rd[q + 1] * (e[q + 1] * e[q + 1]);
            Rd[q] = cdiv(Rl[q] + tt, mk(1.0, 0.0) + Rl[q] * tt);
        }
    }
    cd phx = cexpd(mk(0.0, kx * x));
    cd u = mk(0.0, 0.0);
    if (L == 0) {
        u = phx * cexpd(mk(0.0, -kyv[0].x * y));
    } else {
        // incident wave: down-going in layer 0 with amplitude c at interface 0
        cd c = cexpd(mk(0.0, -kyv[0].x * m.yint[0]));
        if (l == 0) {
            cd inc = c * eikh(kyv[0], -(y - m.yint[0]));          // e^{-i k0y (y - y_0)}
            cd refl = Rd[0] * c * eikh(kyv[0], y - m.yint[0]);    // R~_{01} c e^{i k0y (y - y_0)}
            u = phx * (inc + refl);
        } else {
            // down-going amplitude in layer q, referenced at its top interface
            cd Bq = mk(0.0, 0.0);
            cd prev = c;   // down-going amplitude arriving at the top of the next layer
            for (int q = 1; q <= l; ++q) {
                cd A = m.eta[q - 1] * kyv[q - 1], Bk = m.eta[q] * kyv[q];
                cd Tdn = cdiv(2.0 * A, A + Bk);                              // T_{q-1,q}
                cd den = mk(1.0, 0.0) + Rl[q - 1] * Rd[q] * (e[q] * e[q]);  // 1 - R_{q,q-1} R~_{q,q+1} e^2
                Bq = cdiv(Tdn * prev, den);
                prev = Bq * e[q];
            }
            cd down = Bq * eikh(kyv[l], m.yint[l - 1] - y);
            cd up = mk(0.0, 0.0);
            if (l <= L - 1) up = Rd[l] * Bq * e[l] * eikh(kyv[l], y - m.yint[l]);
            u = phx * (down + up);
        }
    }
    // b = eta_l g, g = -(u_inc + u^b)
    b[t] = -m.eta[l] * u;
}

void rhs_plane_wave_sorted(lfmm_geometry_s* g, int nrhs, const double* angles_host, cd* b_sorted, cudaStream_t s) {
    double* d_ang = nullptr;
    cuda_check(cudaMallocAsync((void**)&d_ang, sizeof(double) * nrhs, s), "malloc angles");
    cuda_check(cudaMemcpyAsync(d_ang, angles_host, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s), "angles h2d");
    int64_t tot = g->n * nrhs;
    k_rhs<<<nblk(tot), 256, 0, s>>>(g->m, g->d_x, g->d_y, g->d_layer, d_ang, nrhs, g->n, b_sorted);
    cuda_check(cudaGetLastError(), "k_rhs");
    cuda_check(cudaStreamSynchronize(s), "rhs");
    cudaFreeAsync(d_ang, s);
}

// ------------------------------------------------------------------ scattered field (eq. integralrep)
// The field is one operator product on a field geometry (elements followed by the m
// field points, which carry weight 0): x = [Phi; 0] per column, and the field-point
// rows of K x are sum_e |Gamma_e| G(c_e, r) Phi_e (or the combined-field kernel).
// x[c (n + m) + i] = Phi[c n + i] (i < n), 0 for the field points; Phi in FP64 or FP32.
__global__ void k_field_pack(const void* __restrict__ phi, int c64, int64_t n, int64_t m, int nrhs,
                             cd* __restrict__ x) {
    const int64_t nm = n + m, tot = nm * nrhs;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = q / nm, i = q - c * nm;
        cd v = mk(0.0, 0.0);
        if (i < n) {
            if (c64) {
                const float2 f = ((const float2*)phi)[c * n + i];
                v = mk((double)f.x, (double)f.y);
            } else {
                v = ((const cd*)phi)[c * n + i];
            }
        }
        x[q] = v;
    }
}
// u[c m + j] = y[c (n + m) + n + j] / eta_{l(r_j)}, in FP64 or rounded to FP32
__global__ void k_field_unpack(const cd* __restrict__ y, const double* __restrict__ inv_eta, int64_t n, int64_t m,
                               int nrhs, int c64, void* __restrict__ u) {
    const int64_t tot = m * nrhs;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = q / m, j = q - c * m;
        const cd v = y[c * (n + m) + n + j] * inv_eta[j];
        if (c64) ((float2*)u)[q] = make_float2((float)v.x, (float)v.y);
        else ((cd*)u)[q] = v;
    }
}

void field_pack(const void* phi, bool c64, int64_t n, int64_t m, int nrhs, cd* x, cudaStream_t s) {
    const int64_t tot = (n + m) * nrhs;
    k_field_pack<<<(int)std::min<int64_t>(nblk(tot), 152 * 16), 256, 0, s>>>(phi, c64 ? 1 : 0, n, m, nrhs, x);
    cuda_check(cudaGetLastError(), "k_field_pack");
}
void field_unpack(const cd* y, const double* inv_eta, int64_t n, int64_t m, int nrhs, bool c64, void* u,
                  cudaStream_t s) {
    const int64_t tot = m * nrhs;
    k_field_unpack<<<(int)std::min<int64_t>(nblk(tot), 152 * 16), 256, 0, s>>>(y, inv_eta, n, m, nrhs, c64 ? 1 : 0,
                                                                                u);
    cuda_check(cudaGetLastError(), "k_field_unpack");
}

}  // namespace lfmm
