// static_scratch.cu -- lfmm_matvec_static: the Nystrom matvec without any allocation.
//
// Some callers cannot allocate device memory at the moment they need a matvec:
// real-time serving threads that must not enter the allocator (cudaMalloc can
// block in the CUDA memory manager and synchronise the device), hosts that
// hand the library a fixed memory budget up front, and frameworks whose own pool
// owns the device memory, where an allocation outside it may fail or fragment.  lfmm_matvec lazily allocates its
// work buffers (sorted copies of x and y, the multipole and local coefficients)
// on first use; this entry point instead uses one file-scope device array of
// fixed size, reserved when the library is loaded.
//
// Properties (also stated in include/lfmm.h):
//  * the array holds LFMM_STATIC_SCRATCH_BYTES (32 MiB) on every GPU that loads
//    the library, until the process exits;
//  * its device address is looked up once per device (cudaGetSymbolAddress, with
//    that device current) on the first call made on that device; make that first
//    call before any stream capture;
//  * every call shares the array, which keeps the last call's contents.  Nothing in
//    it has to start at zero: the sorted output is cleared by the call itself and
//    every coefficient is written before it is read.  Calls that overlap on the GPU
//    (other streams, other threads) race on the array and must be serialised;
//  * geometries whose work buffers do not fit are rejected before any device work.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "geometry.h"

#define LFMM_STATIC_SCRATCH_BYTES (32u << 20)
#define LFMM_STATIC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_static_scratch[LFMM_STATIC_SCRATCH_BYTES];

namespace lfmm {

static std::mutex g_scratch_mutex;
static void* g_scratch_ptr[LFMM_STATIC_MAX_DEVICES] = {};

// Device address of the array on the current device (looked up once per device).
static void* scratch_address() {
    int dev = 0;
    cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= LFMM_STATIC_MAX_DEVICES) throw CudaError{"device index out of range for the static scratch"};
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
        void* ptr = nullptr;
        cuda_check(cudaGetSymbolAddress((void**)&ptr, g_static_scratch), "cudaGetSymbolAddress(static scratch)");
        g_scratch_ptr[dev] = ptr;
    }
    return g_scratch_ptr[dev];
}

static inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace lfmm

using namespace lfmm;

extern "C" lfmm_status lfmm_matvec_static(lfmm_geometry g, const void* x, void* y, void* stream) {
    set_error("");
    if (!g || !x || !y) { set_error("NULL argument"); return LFMM_ERR_INVALID_ARG; }
    if (x == y) { set_error("x and y must not overlap"); return LFMM_ERR_INVALID_ARG; }
    // work buffers: sorted x and y, multipoles/locals (cell centres and reaction centres), M2L partial
    // sums, one column
    const size_t n = (size_t)g->n;
    const size_t b_xs = align256(sizeof(cd) * n), b_ys = b_xs;
    const size_t b_m = align256(sizeof(cd) * (size_t)(g->ncoef > 0 ? g->ncoef : 1));
    const size_t b_mp = align256(sizeof(cd) * (size_t)(g->nslotcoef > 0 ? g->nslotcoef : 1));
    const size_t b_part = align256(sizeof(cd) * (size_t)(g->n_m2l_parts > 0 ? g->n_m2l_parts : 1) * 3 * XT_W);
    const size_t need = b_xs + b_ys + 2 * b_m + 2 * b_mp + b_part;
    if (need > LFMM_STATIC_SCRATCH_BYTES) {
        set_error("geometry needs " + std::to_string(need) + " bytes of work memory; lfmm_matvec_static holds " +
                  std::to_string((size_t)LFMM_STATIC_SCRATCH_BYTES) + " (use lfmm_matvec)");
        return LFMM_ERR_INVALID_ARG;
    }
    // save the geometry's own (lazily allocated) buffers and point it at the array
    cd *sxs = g->d_xs, *sys = g->d_ys, *sM = g->d_M, *sL = g->d_L, *sMp = g->d_Mp, *sLp = g->d_Lp;
    cd* spart = g->d_m2l_part;
    int s_nrhs = g->nrhs_cap, s_cols = g->coef_cols, s_pcols = g->m2l_part_cols;
    bool s_prof = g->prof.on;
    g->prof.on = false;   // the stage timers synchronise the stream; this entry point never does
    lfmm_status st = LFMM_OK;
    try {
        unsigned char* base = (unsigned char*)scratch_address();
        size_t o = 0;
        g->d_xs = (cd*)(base + o); o += b_xs;
        g->d_ys = (cd*)(base + o); o += b_ys;
        g->d_M = (cd*)(base + o); o += b_m;
        g->d_L = (cd*)(base + o); o += b_m;
        g->d_Mp = (cd*)(base + o); o += b_mp;
        g->d_Lp = (cd*)(base + o); o += b_mp;
        g->d_m2l_part = (cd*)(base + o); o += b_part;
        g->nrhs_cap = 1;
        g->coef_cols = 1;
        g->m2l_part_cols = 1;
        cudaStream_t s = (cudaStream_t)stream;
        gather_sorted(g, (const cd*)x, g->d_xs, 1, s);
        apply_operator_sorted(g, g->d_xs, g->d_ys, 1, s);
        scatter_sorted(g, g->d_ys, (cd*)y, 1, s);
    } catch (const CudaError& e) {
        set_error(e.msg);
        st = LFMM_ERR_CUDA;
    } catch (...) {
        set_error("unknown error");
        st = LFMM_ERR_CUDA;
    }
    g->d_xs = sxs; g->d_ys = sys; g->d_M = sM; g->d_L = sL; g->d_Mp = sMp; g->d_Lp = sLp;
    g->d_m2l_part = spart;
    g->nrhs_cap = s_nrhs;
    g->coef_cols = s_cols;
    g->m2l_part_cols = s_pcols;
    g->prof.on = s_prof;
    return st;
}
