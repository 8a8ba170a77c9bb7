// api.cu -- the C ABI (include/lfmm.h): validation, handles, host/device marshalling.
//
// The passages each entry point follows:
//   lfmm_medium_create     Sec. 2.1 (layers between interfaces y = -d_l, wavenumbers k_l,
//                          densities eta_l; eq. TLhelmholtztotallayer1)
//   lfmm_geometry_build    Sec. 3.3 (straight elements collocated at their centres,
//                          eq. linearSystem), Sec. 4.1 (tree and interaction lists, the
//                          moment tables of eq. generalintegral), Sec. 4.2 (the local
//                          matrices of eq. localmatix for the preconditioner)
//   lfmm_rhs_plane_wave    Sec. 2.2 (eqs. incidentwave, homogeneousscattering), scaled as
//                          b = eta g (eq. matrixandvec)
//   lfmm_matvec            eq. Llayerscomponent (Sec. 3.3), the near part stored and the
//                          far part by the FMM of Sec. 4.1
//   lfmm_gmres_solve       Sec. 3.3 (GMRES on eq. EquationSet) with the preconditioner of
//                          Sec. 4.2, tolerance as in Sec. 5
//   lfmm_eval_field        eq. integralrep
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "geometry.h"

namespace lfmm {

static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }

void cuda_check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) throw CudaError{std::string(what) + ": " + cudaGetErrorString(e)};
}

// 8-point Gauss-Legendre rule by Newton iteration on P_8 (no stored tables)
static void gauss_legendre8(double* x, double* w) {
    const int n = 8;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

QuadRule make_quad_rule(const MediumDev& m) {
    QuadRule q;
    q.T = 1.2 * m.kmax + 1.0;
    q.kmin = m.k[0];
    for (int l = 1; l < m.nl; ++l) q.kmin = std::min(q.kmin, m.k[l]);
    q.es_v0 = -3.6;
    q.es_hv = 0.07;
    q.nes = 84;          // v in [-3.6, 2.21]
    q.min_panels = 16;
    // the moment tables' rays: the kernel-value step (a 4x finer step changed no
    // parity figure by more than noise: 5.1e-11, 6.3e-11, 2.7e-10 on three dense
    // checks, C2 rows 2e-10-7e-10, at 1.25x the set-up time)
    q.tab_es_v0 = -3.6;
    q.tab_es_hv = 0.07;
    q.tab_nes = 85;      // v in [-3.6, 2.28]
    // the detour panels of the kernel-value rule plus pS + pT more (the table
    // integrands carry w^n up to |n - m| = 2p); three times as many panels changed
    // neither the wide-band nor the C2 parity (1.2e-10, a few 1e-9) and cost 1.6x
    // the set-up time
    q.tab_panel_mult = 1;
    q.tab_T = table_detour_end(m);
    gauss_legendre8(q.gl_x, q.gl_w);
    return q;
}

void prof_begin(lfmm_geometry_s* g, Stage st, cudaStream_t s) {
    if (!g->prof.on) return;
    cuda_check(cudaEventRecord(g->prof.ev[2 * st], s), "event record");
    g->prof.armed[st] = true;
}
void prof_end(lfmm_geometry_s* g, Stage st, cudaStream_t s) {
    if (!g->prof.on) return;
    cuda_check(cudaEventRecord(g->prof.ev[2 * st + 1], s), "event record");
}
void prof_flush(lfmm_geometry_s* g, cudaStream_t s) {
    if (!g->prof.on) return;
    cuda_check(cudaStreamSynchronize(s), "profile sync");
    for (int k = 0; k < ST_COUNT; ++k) {
        if (!g->prof.armed[k]) continue;
        float ms = 0.f;
        cuda_check(cudaEventElapsedTime(&ms, g->prof.ev[2 * k], g->prof.ev[2 * k + 1]), "event elapsed");
        g->prof.ms[k] += ms;
        g->prof.cnt[k] += 1.0;
        g->prof.armed[k] = false;
    }
}

template <class F>
static lfmm_status guarded_body(F&& f) {
    try {
        t_last_error.clear();
        return f();
    } catch (const ArgError& e) {
        set_error(e.msg);
        return LFMM_ERR_INVALID_ARG;
    } catch (const InterfaceError& e) {
        set_error(e.msg);
        return LFMM_ERR_NODE_ON_INTERFACE;
    } catch (const QuadratureError& e) {
        set_error(e.msg);
        return LFMM_ERR_QUADRATURE;
    } catch (const TimeoutError& e) {
        set_error(e.msg);
        return LFMM_ERR_TIMEOUT;
    } catch (const CudaError& e) {
        set_error(e.msg);
        if (e.msg.find("out of memory") != std::string::npos) return LFMM_ERR_OUT_OF_MEMORY;
        return LFMM_ERR_CUDA;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return LFMM_ERR_OUT_OF_MEMORY;
    } catch (const std::exception& e) {
        set_error(e.what());
        return LFMM_ERR_INVALID_ARG;
    } catch (...) {
        set_error("unknown error");
        return LFMM_ERR_CUDA;
    }
}
// A failed runtime call (an allocation that ran out of memory, say) stays the
// thread's last CUDA error; it is cleared when a call fails, so that the launch
// checks (cudaGetLastError) of the next call on this thread do not report it again.
template <class F>
static lfmm_status guarded(F&& f) {
    const lfmm_status st = guarded_body(std::forward<F>(f));
    if (st < 0) (void)cudaGetLastError();
    return st;
}

lfmm_status guarded_call(const std::function<lfmm_status()>& f) { return guarded(f); }

static void require(bool c, const char* msg) {
    if (!c) throw ArgError{msg};
}

static void free_geometry(lfmm_geometry_s* g) {
    if (g->side) {
        cudaStreamSynchronize(g->side);
        cudaStreamDestroy(g->side);
        g->side = nullptr;
    }
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    g->ev_fork = g->ev_join = nullptr;
    if (g->prof.on)
        for (int k = 0; k < 2 * ST_COUNT; ++k) cudaEventDestroy(g->prof.ev[k]);
    g->prof.on = false;
    fmm_free(g);
    mixed_destroy(g);
    for (void* p : g->allocs) dev_release(p);
    g->allocs.clear();
    dev_release(g->d_xs);
    dev_release(g->d_ys);
    dev_release(g->d_hostbuf_x);
    dev_release(g->d_hostbuf_y);
    dev_release(g->d_near_x32);
    g->d_near_x32 = nullptr;
    g->near_x32_cap = 0;
    cudaStreamSynchronize(cudaStreamPerThread);
}

// sorted-order scratch and host staging for nrhs columns
static void ensure_scratch(lfmm_geometry_s* g, int nrhs) {
    if (g->nrhs_cap < nrhs) {
        dev_release_now(g->d_xs);
        dev_release_now(g->d_ys);
        g->d_xs = g->d_ys = nullptr;
        g->d_xs = (cd*)dev_alloc_ready(sizeof(cd) * g->n * nrhs, "scratch");
        g->d_ys = (cd*)dev_alloc_ready(sizeof(cd) * g->n * nrhs, "scratch");
        g->nrhs_cap = nrhs;
    }
}
static void ensure_hostbuf(lfmm_geometry_s* g, size_t elems) {
    if (g->hostbuf_cap < elems) {
        dev_release_now(g->d_hostbuf_x);
        dev_release_now(g->d_hostbuf_y);
        g->d_hostbuf_x = g->d_hostbuf_y = nullptr;
        g->d_hostbuf_x = (cd*)dev_alloc_ready(sizeof(cd) * elems, "staging");
        g->d_hostbuf_y = (cd*)dev_alloc_ready(sizeof(cd) * elems, "staging");
        g->hostbuf_cap = elems;
    }
}

}  // namespace lfmm

using namespace lfmm;

extern "C" {

const char* lfmm_last_error(void) { return t_last_error.c_str(); }

lfmm_status lfmm_medium_create(int32_t n_layers, const double* interface_y, const double* wavenumber,
                               const double* density, lfmm_medium* out) {
    return guarded([&]() -> lfmm_status {
        require(out != nullptr, "out is NULL");
        require(n_layers >= 1 && n_layers <= LFMM_MAXLAY, "n_layers must be in [1, 16]");
        require(wavenumber != nullptr && density != nullptr, "wavenumber/density is NULL");
        require(n_layers == 1 || interface_y != nullptr, "interface_y is NULL");
        lfmm_medium_s* m = new lfmm_medium_s();
        std::memset(&m->m, 0, sizeof(m->m));
        m->m.nl = n_layers;
        m->m.kmax = 0.0;
        for (int j = 0; j + 1 < n_layers; ++j) {
            double y = interface_y[j];
            if (!std::isfinite(y) || (j > 0 && !(y < interface_y[j - 1]))) {
                delete m;
                throw ArgError{"interface heights must be finite and strictly decreasing"};
            }
            m->m.yint[j] = y;
        }
        for (int l = 0; l < n_layers; ++l) {
            double kr = wavenumber[2 * l], ki = wavenumber[2 * l + 1];
            double eta = density[l];
            if (!(std::isfinite(kr) && kr > 0.0) || ki != 0.0 || !(std::isfinite(eta) && eta > 0.0)) {
                delete m;
                throw ArgError{"wavenumbers must be real and positive (Im k = 0) and densities positive"};
            }
            m->m.k[l] = kr;
            m->m.eta[l] = eta;
            m->m.kmax = std::max(m->m.kmax, kr);
        }
        *out = m;
        return LFMM_OK;
    });
}

lfmm_status lfmm_medium_destroy(lfmm_medium m) {
    return guarded([&]() -> lfmm_status {
        if (!m) return LFMM_OK;
        require(m->geometries == 0, "medium still referenced by a geometry");
        delete m;
        return LFMM_OK;
    });
}

// Builds a geometry; throws on any failure after releasing what it built.  Points with
// input index >= n_src (n_src < n only for the field geometries of lfmm_eval_field) are
// field points: weight 0, never a source, and only the leaves that hold them get near-field
// blocks.
static lfmm_geometry_s* build_geometry(lfmm_medium med, int64_t n, const double* points, const double* weights,
                                       const double* normals, const lfmm_params* prm, int64_t n_src) {
    lfmm_geometry_s* g = nullptr;
    try {
        auto t0 = std::chrono::steady_clock::now();
        require(n >= 1 && n < (int64_t)1 << 31, "n must be in [1, 2^31)");
        require(n_src >= 1 && n_src <= n, "field geometry: bad element count");
        require(points != nullptr && weights != nullptr, "points/weights is NULL");
        int p = prm ? prm->p : 20;
        int leaf = prm ? prm->leaf_size : 64;
        require(p >= 1 && p <= 80, "p must be in [1, 80]");
        require(leaf >= 1 && leaf <= 1024, "leaf_size must be in [1, 1024]");
        const bool cf = prm && (prm->flags & LFMM_COMBINED_FIELD);
        require(!cf || normals != nullptr, "the combined-field operator needs the normals");
        if (cf)
            for (int64_t i = 0; i < n_src; ++i) {
                const double nn = std::hypot(normals[2 * i], normals[2 * i + 1]);
                require(std::isfinite(nn) && std::fabs(nn - 1.0) <= 1e-8, "normals must be unit vectors");
            }
        const MediumDev& m = med->m;
        std::vector<double> px(n), py(n), pw(n);
        std::vector<int> layer(n);
        for (int64_t i = 0; i < n; ++i) {
            px[i] = points[2 * i];
            py[i] = points[2 * i + 1];
            pw[i] = weights[i];
            require(std::isfinite(px[i]) && std::isfinite(py[i]), "points must be finite");
            // element weights are positive; the field points of a field geometry carry weight 0
            require(std::isfinite(pw[i]) && (i < n_src ? pw[i] > 0.0 : pw[i] == 0.0), "weights must be positive");
            int l = 0;
            while (l < m.nl - 1 && py[i] < m.yint[l]) ++l;
            layer[i] = l;
            for (int j = 0; j + 1 < m.nl; ++j) {
                double sc = std::max(1.0, std::fabs(m.yint[j]));
                if (std::fabs(py[i] - m.yint[j]) <= 1e-12 * sc)
                    throw InterfaceError{"a collocation point lies on an interface"};
            }
        }
        g = new lfmm_geometry_s();
        g->n_src = n_src;
        g->med = med;
        g->m = m;
        g->n = n;
        g->p = p;
        g->leaf_size = leaf;
        g->quad = make_quad_rule(m);
        if (prm && (prm->flags & LFMM_PROFILE_STAGES)) {
            for (int k = 0; k < 2 * ST_COUNT; ++k)
                cuda_check(cudaEventCreate(&g->prof.ev[k]), "event create");
            g->prof.on = true;
        }
        auto since = [](std::chrono::steady_clock::time_point a) {
            return std::chrono::duration<double>(std::chrono::steady_clock::now() - a).count();
        };
        auto tp = std::chrono::steady_clock::now();
        {   // the tree and lists on the GPU, from the input points and their layers
            double *d_px = nullptr, *d_py = nullptr;
            int* d_lay = nullptr;
            cudaStream_t ts = cudaStreamPerThread;
            cuda_check(cudaMallocAsync((void**)&d_px, sizeof(double) * n, ts), "malloc points");
            cuda_check(cudaMallocAsync((void**)&d_py, sizeof(double) * n, ts), "malloc points");
            cuda_check(cudaMallocAsync((void**)&d_lay, sizeof(int) * n, ts), "malloc layers");
            struct F {
                double *a, *b;
                int* c;
                ~F() { cudaFreeAsync(a, cudaStreamPerThread); cudaFreeAsync(b, cudaStreamPerThread); cudaFreeAsync(c, cudaStreamPerThread); }
            } fr{d_px, d_py, d_lay};
            cuda_check(cudaMemcpyAsync(d_px, px.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ts), "points");
            cuda_check(cudaMemcpyAsync(d_py, py.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ts), "points");
            cuda_check(cudaMemcpyAsync(d_lay, layer.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ts), "layers");
            build_tree_gpu(g->tree, d_px, d_py, d_lay, n, m, p, leaf);
        }
        g->setup_phase[0] = since(tp);
        TreeHost& t = g->tree;
        if (t.l0 <= t.D) {   // the leaf P2M / L2P stage a group's basis rows in shared memory
            int mx = EXP_GROUP_PTS;
            for (int b = t.level_start[t.D]; b < t.level_start[t.D + 1]; ++b)
                mx = std::max(mx, t.box_end[b] - t.box_begin[b]);
            const size_t pD = (size_t)t.p_level[t.D];
            const size_t p2m = (size_t)mx * (2 * pD + 3) * sizeof(cd) + (size_t)mx * sizeof(cd) + (mx + 1) * sizeof(int);
            const size_t l2p = ((size_t)mx * (pD + 1) + 1) * sizeof(double) + EXP_GROUP_ENTRIES * 2 * (pD + 1) * sizeof(cd);
            require(std::max(p2m, l2p) <= 227 * 1024,
                    "leaf_size too large for the expansion order at the leaves (their P2M / L2P stage a leaf's "
                    "basis rows in shared memory): lower leaf_size or p");
        }
        // sorted-order copies
        g->hx.resize(n); g->hy.resize(n); g->hw.resize(n);
        for (int64_t s = 0; s < n; ++s) {
            int i = t.perm[s];
            g->hx[s] = px[i]; g->hy[s] = py[i]; g->hw[s] = pw[i];
        }
        g->d_x = dupload(g, g->hx);
        g->d_y = dupload(g, g->hy);
        g->d_w = dupload(g, g->hw);
        if (cf) {
            std::vector<double> hnx(n), hny(n);
            for (int64_t s = 0; s < n; ++s) {
                // field points carry no normal (weight 0, never a source)
                hnx[s] = t.perm[s] < n_src ? normals[2 * t.perm[s]] : 1.0;
                hny[s] = t.perm[s] < n_src ? normals[2 * t.perm[s] + 1] : 0.0;
            }
            g->combined = true;
            g->d_nx = dupload(g, hnx);
            g->d_ny = dupload(g, hny);
            g->hnx = std::move(hnx);
            g->hny = std::move(hny);
        }
        g->d_layer = dupload(g, t.layer_sorted);
        g->d_perm = dupload(g, t.perm);
        g->d_box_begin = dupload(g, t.box_begin);
        g->d_box_end = dupload(g, t.box_end);
        g->d_box_layer = dupload(g, t.box_layer);
        g->d_box_level = dupload(g, t.box_level);
        g->d_box_ix = dupload(g, t.box_ix);
        g->d_box_iy = dupload(g, t.box_iy);
        g->d_box_parent = dupload(g, t.box_parent);
        g->d_child_begin = dupload(g, t.child_begin);
        g->d_child_end = dupload(g, t.child_end);
        std::vector<double> bcx(t.nbox), bcy(t.nbox);
        for (int b = 0; b < t.nbox; ++b) { bcx[b] = t.cx(b); bcy[b] = t.cy(b); }
        g->d_box_cx = dupload(g, bcx);
        g->d_box_cy = dupload(g, bcy);
        std::vector<int> comp(4 * std::max<size_t>(t.comps.size(), 1), 0);
        for (size_t c = 0; c < t.comps.size(); ++c) {
            comp[4 * c] = t.comps[c].ls; comp[4 * c + 1] = t.comps[c].a;
            comp[4 * c + 2] = t.comps[c].lt; comp[4 * c + 3] = t.comps[c].b;
        }
        g->d_comp = dupload(g, comp);
        cuda_check(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking), "side stream");
        cuda_check(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming), "event");
        cuda_check(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming), "event");
        tp = std::chrono::steady_clock::now();
        near_build(g);
        g->setup_phase[1] = since(tp);
        tp = std::chrono::steady_clock::now();
        fmm_build(g);
        g->setup_phase[2] = since(tp);
        {   // every stored kernel value and translation table must be finite
            double bad[4];
            count_nonfinite(g, bad);
            if (bad[0] + bad[1] + bad[2] > 0)
                throw QuadratureError{"non-finite values in the stored near field (" + std::to_string((long long)bad[0]) +
                                      "), free-space tables (" + std::to_string((long long)bad[1]) +
                                      ") or reaction tables (" + std::to_string((long long)bad[2]) + ")"};
        }
        if (prm && (prm->flags & LFMM_AUTOTUNE)) fmm_autotune(g);
        g->setup_seconds = since(t0);
        return g;
    } catch (...) {
        if (g) {
            free_geometry(g);
            delete g;
        }
        throw;
    }
}

lfmm_status lfmm_geometry_build(lfmm_medium med, int64_t n, const double* points, const double* weights,
                                const double* normals, const lfmm_params* prm, lfmm_geometry* out) {
    if (out) *out = nullptr;
    return guarded([&]() -> lfmm_status {
        require(med != nullptr && out != nullptr, "medium/out is NULL");
        lfmm_geometry_s* g = build_geometry(med, n, points, weights, normals, prm, n);
        med->geometries += 1;
        *out = g;
        return LFMM_OK;
    });
}

lfmm_status lfmm_geometry_destroy(lfmm_geometry g) {
    return guarded([&]() -> lfmm_status {
        if (!g) return LFMM_OK;
        cudaStreamSynchronize(cudaStreamPerThread);
        free_geometry(g);
        if (g->med) g->med->geometries -= 1;
        delete g;
        return LFMM_OK;
    });
}

static cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

lfmm_status lfmm_matvec(lfmm_geometry g, int32_t nrhs, const void* x, void* y, int32_t flags, void* stream) {
    return guarded([&]() -> lfmm_status {
        require(g != nullptr && x != nullptr && y != nullptr, "NULL argument");
        std::lock_guard<std::mutex> call_lock(g->call_mu);
        require(nrhs >= 1, "nrhs must be >= 1");
        require(x != y, "x and y must not overlap");
        const bool dev = (flags & LFMM_DEVICE_PTRS) != 0;
        const bool c64 = (flags & LFMM_C64) != 0;
        require(!dev || ((uintptr_t)x % 8 == 0 && (uintptr_t)y % 8 == 0), "device vectors must be 8-byte aligned");
        cudaStream_t s = as_stream(stream);
        ensure_scratch(g, nrhs);
        const size_t elems = (size_t)g->n * nrhs;
        const size_t esz = c64 ? sizeof(float2) : sizeof(cd);
        const void* xin = x;
        void* yout = y;
        if (!dev) {
            ensure_hostbuf(g, elems);
            cuda_check(cudaMemcpyAsync(g->d_hostbuf_x, x, esz * elems, cudaMemcpyHostToDevice, s), "x h2d");
            xin = g->d_hostbuf_x;
            yout = g->d_hostbuf_y;
        }
        prof_begin(g, ST_GATHER, s);
        if (c64) gather_sorted_c64(g, (const float2*)xin, g->d_xs, nrhs, s);
        else gather_sorted(g, (const cd*)xin, g->d_xs, nrhs, s);
        prof_end(g, ST_GATHER, s);
        g->m2l_simt = (flags & LFMM_SIMT_M2L) != 0;
        apply_operator_sorted(g, g->d_xs, g->d_ys, nrhs, s, (flags & LFMM_MIXED) != 0);
        g->m2l_simt = false;
        prof_begin(g, ST_SCATTER, s);
        if (c64) scatter_sorted_c64(g, g->d_ys, (float2*)yout, nrhs, s);
        else scatter_sorted(g, g->d_ys, (cd*)yout, nrhs, s);
        prof_end(g, ST_SCATTER, s);
        prof_flush(g, s);
        if (!dev) {
            cuda_check(cudaMemcpyAsync(y, g->d_hostbuf_y, esz * elems, cudaMemcpyDeviceToHost, s), "y d2h");
            cuda_check(cudaStreamSynchronize(s), "matvec sync");
            mixed_check_waits(g);
        }
        return LFMM_OK;
    });
}

lfmm_status lfmm_matvec_batch(int32_t n_geo, const lfmm_geometry* geos, const int32_t* nrhs, const void* const* x,
                              void* const* y, int32_t flags, void* stream) {
    return guarded([&]() -> lfmm_status {
        require(n_geo >= 1 && geos != nullptr && nrhs != nullptr && x != nullptr && y != nullptr, "NULL argument");
        require((flags & LFMM_DEVICE_PTRS) != 0, "lfmm_matvec_batch takes device vectors (LFMM_DEVICE_PTRS)");
        require((flags & ~(LFMM_DEVICE_PTRS | LFMM_C64)) == 0,
                "lfmm_matvec_batch takes LFMM_DEVICE_PTRS, optionally with LFMM_C64, as flags");
        const bool c64 = (flags & LFMM_C64) != 0;
        std::vector<lfmm_geometry_s*> order;
        for (int i = 0; i < n_geo; ++i) {
            require(geos[i] != nullptr && x[i] != nullptr && y[i] != nullptr, "NULL geometry or vector");
            require(nrhs[i] >= 1, "nrhs must be >= 1");
            require(x[i] != y[i], "x and y must not overlap");
            require((uintptr_t)x[i] % 8 == 0 && (uintptr_t)y[i] % 8 == 0, "device vectors must be 8-byte aligned");
            order.push_back(geos[i]);
        }
        std::sort(order.begin(), order.end());
        require(std::adjacent_find(order.begin(), order.end()) == order.end(),
                "a geometry appears twice in the batch");
        // every geometry's lock, in address order (no lock-order inversion between batches)
        std::vector<std::unique_lock<std::mutex>> locks;
        for (lfmm_geometry_s* g : order) locks.emplace_back(g->call_mu);
        cudaStream_t s = as_stream(stream);
        std::vector<BatchOp> ops;
        for (int i = 0; i < n_geo; ++i) {
            lfmm_geometry_s* g = geos[i];
            ensure_scratch(g, nrhs[i]);
            if (c64) gather_sorted_c64(g, (const float2*)x[i], g->d_xs, nrhs[i], s);
            else gather_sorted(g, (const cd*)x[i], g->d_xs, nrhs[i], s);
            ops.push_back(BatchOp{g, g->d_xs, g->d_ys, nrhs[i]});
        }
        apply_operator_batch_sorted(ops, s);
        for (int i = 0; i < n_geo; ++i) {
            lfmm_geometry_s* g = geos[i];
            if (c64) scatter_sorted_c64(g, g->d_ys, (float2*)y[i], nrhs[i], s);
            else scatter_sorted(g, g->d_ys, (cd*)y[i], nrhs[i], s);
        }
        return LFMM_OK;
    });
}

lfmm_status lfmm_precond_apply(lfmm_geometry g, int32_t nrhs, const void* x, void* y, int32_t flags,
                               void* stream) {
    return guarded([&]() -> lfmm_status {
        require(g != nullptr && x != nullptr && y != nullptr, "NULL argument");
        std::lock_guard<std::mutex> call_lock(g->call_mu);
        require(nrhs >= 1, "nrhs must be >= 1");
        require(x != y, "x and y must not overlap");
        require((flags & ~LFMM_DEVICE_PTRS) == 0, "lfmm_precond_apply takes LFMM_DEVICE_PTRS or 0 as flags");
        const bool dev = (flags & LFMM_DEVICE_PTRS) != 0;
        require(!dev || ((uintptr_t)x % 8 == 0 && (uintptr_t)y % 8 == 0), "device vectors must be 8-byte aligned");
        cudaStream_t s = as_stream(stream);
        if (!g->pc_ready) precond_build(g);
        ensure_scratch(g, nrhs);
        const size_t elems = (size_t)g->n * nrhs;
        const void* xin = x;
        void* yout = y;
        if (!dev) {
            ensure_hostbuf(g, elems);
            cuda_check(cudaMemcpyAsync(g->d_hostbuf_x, x, sizeof(cd) * elems, cudaMemcpyHostToDevice, s), "x h2d");
            xin = g->d_hostbuf_x;
            yout = g->d_hostbuf_y;
        }
        gather_sorted(g, (const cd*)xin, g->d_xs, nrhs, s);
        for (int c = 0; c < nrhs; ++c)
            precond_apply_sorted(g, g->d_xs + (size_t)c * g->n, g->d_ys + (size_t)c * g->n, s);
        scatter_sorted(g, g->d_ys, (cd*)yout, nrhs, s);
        if (!dev) {
            cuda_check(cudaMemcpyAsync(y, g->d_hostbuf_y, sizeof(cd) * elems, cudaMemcpyDeviceToHost, s), "y d2h");
            cuda_check(cudaStreamSynchronize(s), "precond sync");
        }
        return LFMM_OK;
    });
}

lfmm_status lfmm_gmres_solve(lfmm_geometry g, int32_t nrhs, const void* b, void* x, const lfmm_gmres_params* prm,
                             lfmm_gmres_info* info, void* stream) {
    return guarded([&]() -> lfmm_status {
        require(g != nullptr && b != nullptr && x != nullptr, "NULL argument");
        std::lock_guard<std::mutex> call_lock(g->call_mu);
        require(nrhs >= 1, "nrhs must be >= 1");
        double tol = prm ? prm->tol : 1e-8;
        int maxit = prm ? prm->max_iter : 1000;
        int pre = prm ? prm->precond : 1;
        const int precision = prm ? prm->precision : 0;
        require(tol > 0.0 && maxit >= 1, "invalid GMRES parameters");
        require(precision == 0 || precision == 1, "precision must be 0 (FP64) or 1 (mixed with refinement)");
        const int restart = prm ? prm->restart : 0;
        require(restart >= 0, "restart must be >= 0 (0 = full GMRES)");
        cudaStream_t s = as_stream(stream);
        if (pre && !g->pc_ready) precond_build(g);
        ensure_scratch(g, nrhs);
        const size_t elems = (size_t)g->n * nrhs;
        cd* bb = nullptr;
        cd* xx = nullptr;
        cuda_check(cudaMallocAsync((void**)&bb, sizeof(cd) * elems, s), "malloc b");
        cuda_check(cudaMallocAsync((void**)&xx, sizeof(cd) * elems, s), "malloc x");
        struct F {
            cd *a, *b;
            cudaStream_t s;
            ~F() { cudaFreeAsync(a, s); cudaFreeAsync(b, s); }
        } fr{bb, xx, s};
        cuda_check(cudaMemcpyAsync(g->d_ys, b, sizeof(cd) * elems, cudaMemcpyDefault, s), "b copy");
        gather_sorted(g, g->d_ys, bb, nrhs, s);
        lfmm_gmres_info local;
        int ok = gmres_sorted(g, bb, xx, nrhs, tol, maxit, pre != 0, s, info ? info : &local, precision,
                              restart);
        scatter_sorted(g, xx, g->d_ys, nrhs, s);
        cuda_check(cudaMemcpyAsync(x, g->d_ys, sizeof(cd) * elems, cudaMemcpyDefault, s), "x copy");
        cuda_check(cudaStreamSynchronize(s), "gmres sync");
        return ok ? LFMM_OK : LFMM_NOT_CONVERGED;
    });
}

lfmm_status lfmm_rhs_plane_wave(lfmm_geometry g, int32_t nrhs, const double* angle_rad, void* b, int32_t flags,
                                void* stream) {
    return guarded([&]() -> lfmm_status {
        require(g != nullptr && angle_rad != nullptr && b != nullptr, "NULL argument");
        std::lock_guard<std::mutex> call_lock(g->call_mu);
        require(nrhs >= 1, "nrhs must be >= 1");
        for (int c = 0; c < nrhs; ++c)
            require(std::isfinite(angle_rad[c]) && angle_rad[c] > 0.0 && angle_rad[c] < M_PI,
                    "incidence angles must lie in (0, pi)");
        const bool dev = (flags & LFMM_DEVICE_PTRS) != 0;
        const bool c64 = (flags & LFMM_C64) != 0;
        require(!dev || (uintptr_t)b % 8 == 0, "device vectors must be 8-byte aligned");
        cudaStream_t s = as_stream(stream);
        ensure_scratch(g, nrhs);
        rhs_plane_wave_sorted(g, nrhs, angle_rad, g->d_xs, s);
        const size_t elems = (size_t)g->n * nrhs;
        void* out = dev ? b : (void*)g->d_ys;
        if (c64) scatter_sorted_c64(g, g->d_xs, (float2*)out, nrhs, s);
        else scatter_sorted(g, g->d_xs, (cd*)out, nrhs, s);
        if (!dev) {
            cuda_check(cudaMemcpyAsync(b, g->d_ys, (c64 ? sizeof(float2) : sizeof(cd)) * elems, cudaMemcpyDeviceToHost,
                                       s), "b d2h");
            cuda_check(cudaStreamSynchronize(s), "rhs sync");
        }
        return LFMM_OK;
    });
}

lfmm_status lfmm_eval_field(lfmm_geometry g, int32_t nrhs, const void* density, int64_t m, const double* targets,
                            void* u, int32_t flags, void* stream) {
    return guarded([&]() -> lfmm_status {
        require(g != nullptr && density != nullptr && targets != nullptr && u != nullptr, "NULL argument");
        std::lock_guard<std::mutex> call_lock(g->call_mu);
        require(nrhs >= 1 && m >= 1, "nrhs and m must be >= 1");
        require(g->n + m < (int64_t)1 << 31, "too many field points");
        const MediumDev& md = g->m;
        std::vector<double> inv_eta(m);
        for (int64_t i = 0; i < m; ++i) {
            require(std::isfinite(targets[2 * i]) && std::isfinite(targets[2 * i + 1]), "targets must be finite");
            int l = 0;
            for (int j = 0; j + 1 < md.nl; ++j) {
                double sc = std::max(1.0, std::fabs(md.yint[j]));
                if (std::fabs(targets[2 * i + 1] - md.yint[j]) <= 1e-12 * sc)
                    throw InterfaceError{"a target lies on an interface"};
                if (targets[2 * i + 1] < md.yint[j]) l = j + 1;
            }
            inv_eta[i] = 1.0 / md.eta[l];
        }
        const bool c64 = (flags & LFMM_C64) != 0;
        cudaStream_t s = as_stream(stream);
        // the field geometry: the elements in their input order, then the field points
        // (weight 0, never a source); same order p, leaf size and operator
        const int64_t n = g->n, nm = g->n + m;
        std::vector<double> pts(2 * nm), wts(nm, 0.0), nrm;
        if (g->combined) nrm.assign(2 * nm, 0.0);
        for (int64_t q = 0; q < n; ++q) {
            const int64_t i = g->tree.perm[q];
            pts[2 * i] = g->hx[q];
            pts[2 * i + 1] = g->hy[q];
            wts[i] = g->hw[q];
            if (g->combined) { nrm[2 * i] = g->hnx[q]; nrm[2 * i + 1] = g->hny[q]; }
        }
        for (int64_t j = 0; j < m; ++j) {
            pts[2 * (n + j)] = targets[2 * j];
            pts[2 * (n + j) + 1] = targets[2 * j + 1];
            if (g->combined) nrm[2 * (n + j)] = 1.0;
        }
        const lfmm_params prm{g->p, g->leaf_size, g->combined ? LFMM_COMBINED_FIELD : 0, 0};
        struct FieldGeometry {
            lfmm_geometry_s* F = nullptr;
            cudaStream_t s;
            ~FieldGeometry() {
                if (!F) return;
                cudaStreamSynchronize(s);
                free_geometry(F);
                delete F;
            }
        } fg{nullptr, s};
        fg.F = build_geometry(g->med, nm, pts.data(), wts.data(), g->combined ? nrm.data() : nullptr, &prm, n);
        lfmm_geometry_s* F = fg.F;
        ensure_scratch(F, nrhs);
        const size_t esz = c64 ? sizeof(float2) : sizeof(cd);
        void* d_phi = nullptr;
        cd* d_xy = nullptr;
        double* d_ie = nullptr;
        void* d_u = nullptr;
        cuda_check(cudaMallocAsync(&d_phi, esz * n * nrhs, s), "malloc density");
        cuda_check(cudaMallocAsync((void**)&d_xy, sizeof(cd) * nm * nrhs, s), "malloc field vector");
        cuda_check(cudaMallocAsync((void**)&d_ie, sizeof(double) * m, s), "malloc 1/eta");
        cuda_check(cudaMallocAsync(&d_u, esz * m * nrhs, s), "malloc u");
        struct Fr {
            void *a, *b, *c, *d;
            cudaStream_t s;
            ~Fr() { cudaFreeAsync(a, s); cudaFreeAsync(b, s); cudaFreeAsync(c, s); cudaFreeAsync(d, s); }
        } fr{d_phi, d_xy, d_ie, d_u, s};
        // density and u may be host or device memory (cudaMemcpyDefault)
        cuda_check(cudaMemcpyAsync(d_phi, density, esz * n * nrhs, cudaMemcpyDefault, s), "density copy");
        cuda_check(cudaMemcpyAsync(d_ie, inv_eta.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s), "1/eta");
        field_pack(d_phi, c64, n, m, nrhs, d_xy, s);
        gather_sorted(F, d_xy, F->d_xs, nrhs, s);
        apply_operator_sorted(F, F->d_xs, F->d_ys, nrhs, s);
        scatter_sorted(F, F->d_ys, d_xy, nrhs, s);
        field_unpack(d_xy, d_ie, n, m, nrhs, c64, d_u, s);
        cuda_check(cudaMemcpyAsync(u, d_u, esz * m * nrhs, cudaMemcpyDefault, s), "u copy");
        cuda_check(cudaStreamSynchronize(s), "field sync");
        return LFMM_OK;
    });
}

lfmm_status lfmm_polygon_elements(int32_t n_poly, const int32_t* counts, const double* vertices, double* points,
                                  double* weights, double* normals) {
    return guarded([&]() -> lfmm_status {
        require(n_poly >= 1 && counts && vertices && points && weights, "NULL or empty argument");
        int64_t base = 0;
        for (int pI = 0; pI < n_poly; ++pI) {
            int nv = counts[pI];
            require(nv >= 3, "a polygon needs at least 3 vertices");
            for (int e = 0; e < nv; ++e) {
                const double* a = vertices + 2 * (base + e);
                const double* b = vertices + 2 * (base + (e + 1) % nv);
                double tx = b[0] - a[0], ty = b[1] - a[1];
                double len = std::hypot(tx, ty);
                require(len > 0.0, "degenerate (zero-length) edge");
                points[2 * (base + e)] = 0.5 * (a[0] + b[0]);
                points[2 * (base + e) + 1] = 0.5 * (a[1] + b[1]);
                weights[base + e] = len;
                if (normals) {
                    normals[2 * (base + e)] = ty / len;
                    normals[2 * (base + e) + 1] = -tx / len;
                }
            }
            base += nv;
        }
        return LFMM_OK;
    });
}

lfmm_status lfmm_geometry_query(lfmm_geometry g, const char* name, void* host_out, int64_t nbytes,
                                int64_t* needed) {
    return guarded([&]() -> lfmm_status {
        require(g != nullptr && name != nullptr, "NULL argument");
        TreeHost& t = g->tree;
        std::vector<int> tmp;
        std::vector<double> dtmp;
        const void* src = nullptr;
        int64_t bytes = 0;
        std::string nm(name);
        auto iv = [&](const std::vector<int>& v) { src = v.data(); bytes = (int64_t)(v.size() * sizeof(int)); };
        if (nm == "perm") iv(t.perm);
        else if (nm == "box_level") iv(t.box_level);
        else if (nm == "box_layer") iv(t.box_layer);
        else if (nm == "box_ix") iv(t.box_ix);
        else if (nm == "box_iy") iv(t.box_iy);
        else if (nm == "box_begin") iv(t.box_begin);
        else if (nm == "box_end") iv(t.box_end);
        else if (nm == "box_parent") iv(t.box_parent);
        else if (nm == "p_level") iv(t.p_level);
        else if (nm == "vfree_ptr") iv(t.vfree_ptr);
        else if (nm == "vfree_idx") iv(t.vfree_idx);
        else if (nm == "ufree_ptr") iv(t.ufree_ptr);
        else if (nm == "ufree_idx") iv(t.ufree_idx);
        else if (nm == "vreact_ptr") iv(t.vreact_ptr);
        else if (nm == "vreact_idx") iv(t.vreact_idx);
        else if (nm == "vreact_comp") iv(t.vreact_comp);
        else if (nm == "ureact_ptr") iv(t.ureact_ptr);
        else if (nm == "ureact_idx") iv(t.ureact_idx);
        else if (nm == "ureact_comp") iv(t.ureact_comp);
        else if (nm == "components") {
            for (auto& c : t.comps) { tmp.push_back(c.ls); tmp.push_back(c.a); tmp.push_back(c.lt); tmp.push_back(c.b); }
            iv(tmp);
        } else if (nm == "tree_params") {
            dtmp = {t.x0, t.y0, t.W, (double)t.D, (double)t.l0, (double)t.nbox, (double)t.comps.size(),
                    (double)g->n_blocks, (double)g->nb_nnz, (double)g->n_rkeys, g->setup_seconds};
            src = dtmp.data();
            bytes = (int64_t)(dtmp.size() * sizeof(double));
        } else if (nm == "near_entries") {
            dtmp = {(double)g->nb_nnz, (double)g->near32_nnz, (double)g->near64r_nnz};
            src = dtmp.data();
            bytes = (int64_t)(dtmp.size() * sizeof(double));
        } else if (nm == "setup_times") {
            dtmp = {g->setup_phase[0], g->setup_phase[1], g->setup_phase[2], g->setup_seconds};
            src = dtmp.data();
            bytes = (int64_t)(dtmp.size() * sizeof(double));
        } else if (nm == "nonfinite") {
            dtmp.assign(4, 0.0);
            count_nonfinite(g, dtmp.data());
            src = dtmp.data();
            bytes = (int64_t)(dtmp.size() * sizeof(double));
        } else if (nm == "reaction_tables") {
            react_key_report(g, dtmp);
            src = dtmp.data();
            bytes = (int64_t)(dtmp.size() * sizeof(double));
        } else if (nm == "table_work") {
            dtmp = {g->table_cmacs[0], g->table_cmacs[1]};
            src = dtmp.data();
            bytes = (int64_t)(dtmp.size() * sizeof(double));
        } else if (nm == "precision_form") {
            int lm = 0, df = 0;
            double rg[3];
            mixed_info(g, &lm, &df, rg);
            dtmp = {(double)lm, (double)df, rg[0], rg[1], rg[2]};
            src = dtmp.data();
            bytes = (int64_t)(dtmp.size() * sizeof(double));
        } else if (nm == "launch_count") {
            dtmp = {(double)g->n_launches};
            src = dtmp.data();
            bytes = (int64_t)sizeof(double);
        } else if (nm == "tuning") {
            dtmp = {(double)g->m2l_item_work, (double)g->m2l_wide, g->tune_ms_default, g->tune_ms_best};
            src = dtmp.data();
            bytes = (int64_t)(dtmp.size() * sizeof(double));
        } else if (nm == "stage_times") {
            for (int k = 0; k < ST_COUNT; ++k) { dtmp.push_back(g->prof.cnt[k]); dtmp.push_back(g->prof.ms[k]); }
            src = dtmp.data();
            bytes = (int64_t)(dtmp.size() * sizeof(double));
        } else {
            throw ArgError{"unknown query name"};
        }
        if (needed) *needed = bytes;
        if (host_out && nbytes >= bytes && bytes > 0) std::memcpy(host_out, src, (size_t)bytes);
        return LFMM_OK;
    });
}

}  // extern "C"
