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
//  * geometries whose work buffers do not fit are rejected before any device work;
//  * for the length of the call the geometry's work-buffer fields point into the
//    array, under the geometry's call lock, which every other entry point that
//    applies the operator also takes: a concurrent lfmm_matvec, lfmm_gmres_solve,
//    lfmm_eval_field or server worker on the same geometry waits on the host instead
//    of enqueueing work on the array.  Work already enqueued on another stream is
//    not waited for: the caller orders the streams it uses with one geometry.
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

// The geometry's work-buffer fields, pointed at the static array for the length of one
// call and restored when the call ends (also when it throws).
struct ScratchSwap {
    lfmm_geometry_s* g;
    cd *xs, *ys, *M, *L, *Mp, *Lp, *part;
    int nrhs_cap, coef_cols, part_cols;
    bool prof;
    explicit ScratchSwap(lfmm_geometry_s* geo)
        : g(geo), xs(geo->d_xs), ys(geo->d_ys), M(geo->d_M), L(geo->d_L), Mp(geo->d_Mp), Lp(geo->d_Lp),
          part(geo->d_m2l_part), nrhs_cap(geo->nrhs_cap), coef_cols(geo->coef_cols),
          part_cols(geo->m2l_part_cols), prof(geo->prof.on) {}
    ~ScratchSwap() {
        g->d_xs = xs; g->d_ys = ys; g->d_M = M; g->d_L = L; g->d_Mp = Mp; g->d_Lp = Lp;
        g->d_m2l_part = part;
        g->nrhs_cap = nrhs_cap;
        g->coef_cols = coef_cols;
        g->m2l_part_cols = part_cols;
        g->prof.on = prof;
    }
};

}  // namespace lfmm

using namespace lfmm;

extern "C" lfmm_status lfmm_matvec_static(lfmm_geometry g, const void* x, void* y, void* stream) {
    return guarded_call([&]() -> lfmm_status {
        if (!g || !x || !y) throw ArgError{"NULL argument"};
        if (x == y) throw ArgError{"x and y must not overlap"};
        if ((uintptr_t)x % 8 != 0 || (uintptr_t)y % 8 != 0) throw ArgError{"device vectors must be 8-byte aligned"};
        // work buffers: sorted x and y, multipoles/locals (cell centres and reaction centres), M2L
        // partial sums, one column
        const size_t n = (size_t)g->n;
        const size_t b_xs = align256(sizeof(cd) * n), b_ys = b_xs;
        const size_t b_m = align256(sizeof(cd) * (size_t)(g->ncoef > 0 ? g->ncoef : 1));
        const size_t b_mp = align256(sizeof(cd) * (size_t)(g->nslotcoef > 0 ? g->nslotcoef : 1));
        const size_t b_part = align256(sizeof(cd) * (size_t)(g->n_m2l_parts > 0 ? g->n_m2l_parts : 1) * 3 * XT_W);
        const size_t need = b_xs + b_ys + 2 * b_m + 2 * b_mp + b_part;
        if (need > LFMM_STATIC_SCRATCH_BYTES)
            throw ArgError{"geometry needs " + std::to_string(need) + " bytes of work memory; lfmm_matvec_static holds " +
                           std::to_string((size_t)LFMM_STATIC_SCRATCH_BYTES) + " (use lfmm_matvec)"};
        // other calls on this geometry wait while its buffer fields point at the array
        std::lock_guard<std::mutex> call_lock(g->call_mu);
        unsigned char* base = (unsigned char*)scratch_address();
        ScratchSwap keep(g);
        g->prof.on = false;   // the stage timers synchronise the stream; this entry point never does
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
        return LFMM_OK;
    });
}
