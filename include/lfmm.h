/*
 * lfmm.h -- C ABI of the layered-medium fast multipole boundary-integral solver.
 *
 * The library solves 2-D sound-soft acoustic scattering by many bodies in a
 * medium of horizontal layers with the single-layer, first-kind boundary
 * integral equation of Sec. 3 of the paper (eqs. integralrep and
 * BoundaryIntergateEquation), discretised by the lowest-order Nystrom method
 * (eqs. linearSystem, matrixelmemts).  The operator K is applied by a fast
 * multipole method with a free-space part per layer and reaction parts per
 * non-zero reaction component (Sec. 4.1), the system K Phi = b is solved by
 * GMRES with the overlapping domain-decomposition preconditioner of Sec. 4.2.
 *
 * Conventions shared by every call
 *  - All functions are extern "C", never throw, and return an lfmm_status.
 *    On error, lfmm_last_error() returns a thread-local message valid until
 *    the next call on the same thread.  Argument errors are reported before
 *    any device work, except lfmm_geometry_build's check of the leaf size
 *    against the order at the leaves, which needs the tree (built on the GPU).
 *  - Complex vectors are interleaved (re, im) double precision (single
 *    precision with LFMM_C64, where a call takes flags), column-major
 *    [n x nrhs] (column j starts at element j*n).  Device vectors must be
 *    8-byte aligned.
 *  - The unknown is the paper's Phi = eta * phi and the right-hand side is
 *    b = eta_{l'} g (Sec. 3.3, eq. matrixandvec); element order is the order
 *    of the points passed to lfmm_geometry_build.
 *  - Vector pointers are HOST pointers unless flags contain LFMM_DEVICE_PTRS,
 *    in which case they are device pointers valid on `stream`.  `stream` is a
 *    cudaStream_t (NULL = the legacy default stream).  Calls with host
 *    pointers synchronise the stream before returning.
 *  - Ownership: input arrays are borrowed for the duration of the call and
 *    copied; outputs are caller allocated.  Handles are owned by the library
 *    until the matching _destroy.  A geometry keeps a reference to its medium:
 *    destroying a medium that still has geometries is refused.
 *  - Thread safety: calls on different geometries may run concurrently.  Calls
 *    on one geometry take the geometry's lock, so calls from several threads
 *    enqueue their work one after another; device work they enqueue on
 *    different streams is not ordered by the library, so a caller using one
 *    geometry from several streams orders those streams itself.
 */
#ifndef LFMM_H
#define LFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LFMM_OK = 0,
    LFMM_NOT_CONVERGED = 1,           /* warning: outputs are valid (best iterate) */
    LFMM_ERR_INVALID_ARG = -1,
    LFMM_ERR_OUT_OF_MEMORY = -2,
    LFMM_ERR_CUDA = -3,
    LFMM_ERR_NODE_ON_INTERFACE = -4,  /* a point lies on (or within 1e-12*scale of) an interface */
    LFMM_ERR_QUADRATURE = -5,         /* lfmm_geometry_build: a stored near-field value or a
                                         translation table came out non-finite (checked at the
                                         end of every build); the quadrature rules are fixed, so
                                         this marks a medium or order beyond their range */
    LFMM_ERR_TIMEOUT = -6,            /* a bounded device wait gave up: the tensor-core
                                         M2L of LFMM_MIXED (16+ columns) waits on its own
                                         MMAs.  The affected products were computed with
                                         those M2L contributions zeroed.  A call with host
                                         vectors reports it itself; with device vectors the
                                         next lfmm_matvec on the geometry does.  Reported
                                         once, after which the geometry is usable again */
    LFMM_ERR_HBM_BUDGET = -7
} lfmm_status;

enum {
    LFMM_DEVICE_PTRS = 1,   /* vector arguments are device pointers */
    LFMM_MIXED = 2          /* lfmm_matvec: apply the precision form of the operator --
                               the far field (P2M, M2M, M2L free space and reaction, L2L,
                               L2P) in FP32 on scaled expansions on the levels whose order
                               is at most 1.5 p, and the regular near field (stored blocks
                               that hold only free-space entries) in complex64 with FP32
                               products.  FP64 stays for the coarser wide-band levels, the
                               self terms I^s, the near blocks that hold reaction
                               (Sommerfeld) entries and every sum into y.  Its relative
                               difference from the FP64 operator is a few 1e-7 (no
                               counterpart in the paper, which works in FP64 throughout).
                               The complex64 near field is built on the first such call.
                               With 16 or more columns its M2L runs on the tensor cores
                               (3xTF32, tcgen05) */,
    LFMM_SIMT_M2L = 8,      /* with LFMM_MIXED: keep the FP32 M2L on the SIMT kernel for
                               any number of columns (same operator to FP32 rounding) */
    LFMM_C64 = 16           /* lfmm_matvec, lfmm_rhs_plane_wave, lfmm_eval_field: the complex
                               vector arguments are single precision (interleaved float re,
                               im; same column-major layout).  They are widened to FP64 on the
                               device, the call computes exactly as without the flag, and its
                               outputs are rounded to the nearest single-precision value.
                               Halves the vectors' host-device traffic.  lfmm_gmres_solve
                               takes double-precision vectors only */
};

/* lfmm_params.flags */
enum {
    LFMM_PROFILE_STAGES = 1 /* time every stage of lfmm_matvec with CUDA events on the call's
                               stream (adds one stream synchronisation per call); read the
                               totals with lfmm_geometry_query("stage_times") */,
    LFMM_AUTOTUNE = 2       /* choose the schedule of the M2L work items (cap on the work of
                               one item, one row per narrow box or not) by timing the
                               candidates on this geometry at set-up (some 40 M2L launches);
                               read the choice with lfmm_geometry_query("tuning").  Results
                               differ from the default schedule only in the order in which
                               the parts of a split sum are added */,
    LFMM_COMBINED_FIELD = 4 /* combined-field operator instead of the paper's single layer
                               (needs the normals): 1/2 I + D - i k S with D the double
                               layer of the layered Green's function (normal derivative at
                               the element, outward normals) and the coupling k of the
                               element's layer; the unknown, the right-hand side and the
                               field keep their single-layer meaning otherwise.  Second
                               kind: GMRES iterations stay nearly flat under refinement */
};

typedef struct lfmm_medium_s *lfmm_medium;
typedef struct lfmm_geometry_s *lfmm_geometry;

/* FMM parameters (NULL = defaults). */
typedef struct {
    int32_t p;          /* expansion order at the fine levels (default 20); coarse levels
                           raise it with k*w (wide-band rule), up to 80 */
    int32_t leaf_size;  /* max points per leaf box (default 64) */
    int32_t flags;      /* LFMM_PROFILE_STAGES | LFMM_AUTOTUNE | LFMM_COMBINED_FIELD, or 0 */
    int32_t reserved;
} lfmm_params;

/* GMRES parameters (NULL = defaults). */
typedef struct {
    double tol;         /* relative residual ||b - K x|| / ||b|| (default 1e-8, Sec. 5) */
    int32_t max_iter;   /* default 1000 */
    int32_t restart;    /* 0 = full GMRES (default).  m > 0: GMRES(m): a pass builds at
                           most m Krylov vectors for the correction of the residual
                           b - K x, which is recomputed with the FP64 operator before the
                           next pass; max_iter counts the steps of all passes.  Bounds the
                           Krylov basis to (m + 1) n complex values per column.  Columns are
                           then solved one after another */
    int32_t precond;    /* 1 = overlapping DD preconditioner (Sec. 4.2, default), 0 = none */
    int32_t precision;  /* 0 = FP64 operator (default); if the residual recomputed after
                           full GMRES misses tol (rounding drift of a long run), refinement
                           passes on b - K x follow while steps remain.  1 = relaxed mixed
                           precision:
                           the relative difference eps of the LFMM_MIXED and FP64
                           operators is measured on b; GMRES multiplies by the FP64
                           operator until its residual falls below 0.03 tol / eps and by
                           the LFMM_MIXED one after that, to 0.3 tol; the FP64 residual is then
                           recomputed and refinement steps run while it exceeds tol.
                           tol applies to that FP64 residual */
} lfmm_gmres_params;

typedef struct {
    int32_t iterations;        /* Krylov iterations of the last right-hand side */
    int32_t converged;         /* 1 if every column reached tol */
    double rel_residual;       /* final GMRES residual estimate (max over columns) */
    double true_rel_residual;  /* ||b - K x|| / ||b|| recomputed with lfmm_matvec (max over columns) */
    double solve_seconds;      /* wall time of the solve */
    int32_t refinements;       /* GMRES passes of the last column after the first: restart
                                  cycles and refinement steps (full FP64 GMRES: 0, unless the
                                  recomputed residual missed tol and refinement passes ran) */
    int32_t fp64_matvecs;      /* FP64 operator applications, Krylov steps and residuals
                                  (last column) */
    double op_rel_diff;        /* precision 1: ||(A_mixed - A) b|| / ||A b|| (max over columns),
                                  the operator difference the relaxation was set from */
} lfmm_gmres_info;

/*
 * Layered medium (Sec. 2.1).  n_layers = L+1 >= 1 layers, top layer first.
 *   interface_y : L interface heights y = -d_l, strictly decreasing
 *   wavenumber  : 2*(L+1) doubles, complex k_l (re, im); Re k > 0.  The library
 *                 supports real wavenumbers only (Im k must be 0).
 *   density     : L+1 values eta_l > 0 (the paper's "reflection index")
 * Errors: LFMM_ERR_INVALID_ARG for any violated condition.
 */
lfmm_status lfmm_medium_create(int32_t n_layers, const double *interface_y,
                               const double *wavenumber, const double *density,
                               lfmm_medium *out);
lfmm_status lfmm_medium_destroy(lfmm_medium m);

/*
 * Discretised scatterer boundaries (Sec. 3.3) and everything the fast
 * operator needs: layer of each point, quadtree and interaction lists,
 * Sommerfeld tables and near-field blocks, the preconditioner.
 *   n       : number of elements/collocation points (>= 1)
 *   points  : 2n doubles, collocation points (x, y) (element centres)
 *   weights : n doubles, element lengths |Gamma_e| > 0
 *   normals : 2n doubles, outward unit normals (needed with LFMM_COMBINED_FIELD,
 *             else NULL or ignored)
 *   prm     : NULL for defaults
 * Errors: LFMM_ERR_INVALID_ARG, LFMM_ERR_NODE_ON_INTERFACE, LFMM_ERR_OUT_OF_MEMORY,
 *         LFMM_ERR_CUDA; *out is then NULL and whatever was built is released.
 */
lfmm_status lfmm_geometry_build(lfmm_medium m, int64_t n, const double *points,
                                const double *weights, const double *normals,
                                const lfmm_params *prm, lfmm_geometry *out);
/* Releases the geometry's device memory (stream-ordered, without a device-wide
 * synchronisation): synchronise every stream passed to calls on it first. */
lfmm_status lfmm_geometry_destroy(lfmm_geometry g);

/*
 * Right-hand side of a plane incident wave (Sec. 2.2): b = eta_{l'} g with
 * g = -(u_inc + u^b) on boundaries in the top layer and -u^b below
 * (eq. homogeneousscattering); u_inc = exp(i k0 (x cos a - y sin a)) in the top
 * layer, a in (0, pi) measured from the +x axis; u^b the background field.
 *   nrhs      : number of incidence angles (columns of b)
 *   angle_rad : nrhs angles (host array)
 *   b         : [n x nrhs] complex output
 */
lfmm_status lfmm_rhs_plane_wave(lfmm_geometry g, int32_t nrhs, const double *angle_rad,
                                void *b, int32_t flags, void *stream);

/*
 * y = K x, the Nystrom matrix-vector product of eq. Llayerscomponent (Sec. 3.3),
 * applied by the layered-medium FMM (Sec. 4.1).  x and y: [n x nrhs] complex.
 * x and y must not overlap.
 */
lfmm_status lfmm_matvec(lfmm_geometry g, int32_t nrhs, const void *x, void *y,
                        int32_t flags, void *stream);

/*
 * y_i = K_i x_i for n_geo geometries at once (no counterpart in the paper, which
 * treats one problem at a time): each stage of the operator -- near field, P2M,
 * every M2M pass, M2L with its reductions, every L2L pass, L2P -- runs as one
 * launch whose blocks cover all the geometries' work, so many small or uneven
 * problems fill the GPU together.  Each y_i equals lfmm_matvec(geos[i], nrhs[i],
 * x[i], y_i) bit for bit (the same kernel bodies sum in the same order).
 *   geos : n_geo distinct geometries (one may not appear twice)
 *   nrhs : n_geo column counts; x[i], y[i] : [n_i x nrhs[i]] DEVICE vectors
 *          (flags must contain LFMM_DEVICE_PTRS; LFMM_C64 for complex64
 *          vectors, widened and rounded as in lfmm_matvec), valid on `stream`
 * The FP64 operator (LFMM_MIXED is not taken).  Holds every geometry's lock for
 * the call.  Errors: LFMM_ERR_INVALID_ARG for NULL or overlapping vectors, other
 * flags, a repeated geometry, nrhs < 1, misaligned vectors; LFMM_ERR_CUDA,
 * LFMM_ERR_OUT_OF_MEMORY from the work buffers.
 */
lfmm_status lfmm_matvec_batch(int32_t n_geo, const lfmm_geometry *geos, const int32_t *nrhs,
                              const void *const *x, void *const *y, int32_t flags, void *stream);

/*
 * y = P^{-1} x, the overlapping domain-decomposition preconditioner of Sec. 4.2
 * alone (the operator lfmm_gmres_solve applies on the right when prm->precond
 * is set).  For every leaf box B of every layer's tree, P_B is the local matrix
 * of eq. localmatix on the points of B and of its same-layer neighbour leaves
 * (the free-space Nystrom entries with the self terms I^s on the diagonal); only
 * the rows of P_B^{-1} that belong to B's own points are kept (restricted
 * additive Schwarz), so y_B = (P_B^{-1} x_J)|_B.  Built on first use (one LU
 * per leaf).  x and y: [n x nrhs] complex128 in host memory, or device memory
 * with flags = LFMM_DEVICE_PTRS; they must not overlap.  Errors:
 * LFMM_ERR_INVALID_ARG (NULL, nrhs < 1, x == y, other flags, misaligned device
 * vectors); LFMM_ERR_CUDA or LFMM_ERR_OUT_OF_MEMORY from the set-up.
 */
lfmm_status lfmm_precond_apply(lfmm_geometry g, int32_t nrhs, const void *x, void *y,
                               int32_t flags, void *stream);

/*
 * y = K x like lfmm_matvec (one right-hand side, DEVICE pointers on `stream`),
 * but allocating nothing.  The paper has no counterpart: this exists for
 * callers that cannot allocate device memory when they need a matvec --
 * real-time threads that must stay out of the allocator (an allocation can block
 * and synchronise the device), hosts with a fixed memory budget, frameworks whose
 * own pool owns the device memory.  lfmm_matvec
 * allocates its work buffers on first use; this call uses instead one
 * file-scope device array of 32 MiB that every GPU loading the library holds
 * until the process exits.
 *   - The array's device address is looked up on the first call made on each
 *     device (with that device current); make that first call before any
 *     stream capture.
 *   - All calls share the array and it keeps the last call's contents; calls
 *     that overlap on the GPU (other streams or threads) race and must be
 *     serialised by the caller.
 *   - While the call runs, the geometry's work-buffer fields point into the
 *     array.  It holds the geometry's lock meanwhile, so another thread's call
 *     on the same geometry (lfmm_matvec, lfmm_gmres_solve, ...) waits; work
 *     such calls enqueued earlier on other streams must have finished (the
 *     caller orders the streams).
 *   - Errors: LFMM_ERR_INVALID_ARG for NULL, overlapping or not 8-byte aligned
 *     vectors and for geometries whose work buffers do not fit (y is then left
 *     untouched); LFMM_ERR_CUDA for a failed launch.
 *   - Geometries whose work buffers (sorted x and y, multipole and local
 *     coefficients, M2L partial sums) exceed the array are rejected with LFMM_ERR_INVALID_ARG
 *     before any device work (C2-sized problems, N = 65536, need about 16 MiB).
 *   - The stage profiler is not run by this call; the operator is the FP64 one.
 */
lfmm_status lfmm_matvec_static(lfmm_geometry g, const void *x, void *y, void *stream);

/*
 * Solve K x = b by GMRES (x0 = 0), right-preconditioned by the overlapping
 * domain-decomposition preconditioner when prm->precond is set (Sec. 4.2).
 * Several columns with the FP64 operator and full GMRES (restart 0) advance
 * together -- one Krylov space per column, every step one block matvec of the
 * active columns -- when their bases fit in a quarter of the free device memory;
 * each column's result equals its separate solve.  Otherwise columns are solved
 * one after another.  b and x are complex128, in host or device memory.  Returns
 * LFMM_NOT_CONVERGED (with the best iterate in x and info filled) if max_iter is
 * reached.
 */
lfmm_status lfmm_gmres_solve(lfmm_geometry g, int32_t nrhs, const void *b, void *x,
                             const lfmm_gmres_params *prm, lfmm_gmres_info *info,
                             void *stream);

/*
 * Scattered field u^s at m off-boundary targets from the density Phi
 * (eq. integralrep):  u^s(r) = (1/eta_{l(r)}) sum_e Phi_e |Gamma_e| G_{l_e l(r)}(c_e, r).
 *   density : [n x nrhs] complex Phi (host or device memory)
 *   targets : 2m doubles (host)
 *   u       : [m x nrhs] complex output (host or device memory)
 *   flags   : LFMM_C64 for single-precision density and u, else 0
 * The field is evaluated through the same expansions as lfmm_matvec: the call
 * builds a field geometry -- the elements followed by the m targets, which carry
 * weight 0 and are never sources -- with the geometry's order p, leaf size and
 * operator, and takes the targets' rows of one FMM product with [Phi; 0]
 * (far field by P2M, M2M, M2L, L2L, L2P; near field by the stored free-space and
 * Sommerfeld entries, built only for leaves that hold targets).  Cost: one
 * geometry set-up over n + m points plus one product, instead of m n Sommerfeld
 * integrals; every sum has a fixed order, so repeated calls give the same bits.
 * Targets must lie off the boundary (a target at an element centre meets the
 * kernel's singularity).  A target on an interface returns
 * LFMM_ERR_NODE_ON_INTERFACE.  Synchronises the stream.
 */
lfmm_status lfmm_eval_field(lfmm_geometry g, int32_t nrhs, const void *density, int64_t m,
                            const double *targets, void *u, int32_t flags, void *stream);

/*
 * Elements of closed counter-clockwise polygons (Sec. 3.3: straight elements,
 * collocation at the element centre).  Host-only helper.
 *   n_poly, counts : number of polygons and vertices per polygon
 *   vertices       : concatenated (x, y) vertices
 *   points, weights, normals : outputs (2N, N, 2N doubles), N = sum(counts);
 *                    chord midpoints, chord lengths, outward unit normals
 */
lfmm_status lfmm_polygon_elements(int32_t n_poly, const int32_t *counts, const double *vertices,
                                  double *points, double *weights, double *normals);

/*
 * Serving: a request loop for scattering solves (no counterpart in the paper,
 * which solves one problem at a time).  Requests -- a layer stack, scatterer
 * elements, one incidence angle, a tolerance and the precision -- queue in
 * arrival order.  `slots` worker threads each drive one CUDA stream on the
 * current device; a worker takes the request at the head of the queue as soon as
 * the estimated device footprints of the running requests plus this one fit
 * hbm_budget, and runs it end to end (lfmm_medium_create, lfmm_geometry_build,
 * lfmm_rhs_plane_wave, lfmm_gmres_solve, copy of the solution, release).
 * Requests that arrive while others run are admitted as slots and memory free
 * up; their kernels overlap on the device.  Every kernel sums in a fixed order
 * and each request has its own geometry and Krylov basis, so a result is the
 * same alone and in the mix.
 *   footprint estimate (bytes): 16 n (max_iter + 1) for the Krylov basis, plus
 *   about 16 n (120 (1 + leaf/64) + 24) for near field, preconditioner and work
 *   vectors, 4 n (2p + 1) for expansions, and 256 MiB for tables and scratch.
 */
typedef struct lfmm_server_s *lfmm_server;
typedef struct {
    int32_t slots;        /* concurrent requests (worker threads, one stream each), 1..64 */
    int32_t reserved;
    int64_t hbm_budget;   /* device bytes the running requests' footprints may total */
} lfmm_server_params;
typedef struct {
    int32_t n_layers;            /* as lfmm_medium_create */
    int32_t p;                   /* expansion order (<= 0: 20) */
    const double *interface_y;   /* n_layers - 1 values */
    const double *wavenumber;    /* 2 n_layers (re, im) */
    const double *density;       /* n_layers */
    int64_t n;                   /* elements */
    const double *points;        /* 2n, host */
    const double *weights;       /* n, host */
    double angle_rad;            /* plane-wave incidence, (0, pi) */
    double tol;                  /* GMRES relative residual (FP64 residual) */
    int32_t precision;           /* 0: FP64 operator; 1: relaxed mixed precision */
    int32_t leaf_size;           /* <= 0: 64 */
    int32_t max_iter;
    int32_t precond;             /* 1: DD preconditioner */
    const double *normals;       /* 2n outward unit normals, host; needed with LFMM_COMBINED_FIELD */
    int32_t flags;               /* 0 or LFMM_COMBINED_FIELD (the geometry's operator) */
    int32_t reserved;
} lfmm_request;                  /* every array is copied by lfmm_server_submit */
typedef struct {
    double queue_seconds;        /* submit -> admitted */
    double service_seconds;      /* admitted -> solution in host memory */
    double latency_seconds;      /* submit -> solution in host memory */
    double setup_seconds;        /* geometry build inside the service time */
    int64_t footprint_bytes;     /* the estimate admission used */
} lfmm_request_times;

/* Errors: LFMM_ERR_INVALID_ARG; LFMM_ERR_CUDA if no device is current. */
lfmm_status lfmm_server_create(const lfmm_server_params *prm, lfmm_server *out);
/* Queue a request; *ticket identifies it.  LFMM_ERR_HBM_BUDGET if its footprint
 * estimate alone exceeds the budget (it could never be admitted). */
lfmm_status lfmm_server_submit(lfmm_server s, const lfmm_request *req, int64_t *ticket);
/* Block until the request is done; x (host, n complex) receives the solution Phi,
 * info and times (either may be NULL) its GMRES record and timings.  Returns the
 * request's status (the solve's, or the first error of its pipeline). */
lfmm_status lfmm_server_wait(lfmm_server s, int64_t ticket, void *x, lfmm_gmres_info *info,
                             lfmm_request_times *times);
/* Largest total footprint admitted at once and largest number of requests run at once. */
lfmm_status lfmm_server_stats(lfmm_server s, int64_t *peak_bytes, int32_t *peak_running);
/* Runs the queued requests to completion, then stops the workers. */
lfmm_status lfmm_server_destroy(lfmm_server s);

/*
 * Introspection of a built geometry (used by the tests).  Copies the named
 * array to host memory: `needed` receives its size in bytes; if host_out is
 * NULL or nbytes is too small nothing is copied.  Names: "perm" (int32[n],
 * sorted position -> input index), "box_level", "box_layer", "box_ix",
 * "box_iy", "box_begin", "box_end", "box_parent" (int32[nbox]),
 * "tree_params" (double[11]: x0, y0, W, D, l0, nbox, ncomp, n_near_blocks,
 * near-field entries, reaction M2L tables, set-up seconds),
 * "stage_times" (double[2*8]: per stage p2m, m2m, m2l, l2l, l2p, near, gather,
 * scatter the number of timed launches and their total milliseconds),
 * "near_entries" (double[3]: stored near-field entries of the FP64 operator; of the
 * precision form, entries held in complex64 and in FP64 -- 0 until its first call),
 * "setup_times" (double[4]: seconds of the set-up spent on the tree and interaction
 * lists, the near field, the far field (moment tables, translation plans), and in all),
 * "nonfinite" (double[4]: non-finite entries of the stored near field, the free-space and
 * reaction translation tables, and the preconditioner once built -- all 0 for a sound geometry),
 * "reaction_tables" (double[8 * tables]: per reaction moment table its component, level,
 * order, horizontal offset X, source and target heights, effective distance D and its
 * non-finite entries),
 * "table_work" (double[2]: complex multiply-adds of the set-up's reaction moment tables,
 * cross-layer and same-layer components: entries x quadrature nodes x 2),
 * "precision_form" (double[5]: first level of the precision form's FP32 far field;
 * 1 if its coarser levels' M2L runs in double-float, 0 if in FP64, -1 before its first call;
 * log10 of the largest free-space and reaction table component of those levels and of their
 * largest scaled multipole basis value -- double-float needs their sums to stay at most 26),
 * "launch_count" (double[1]: kernels launched so far by this geometry's
 * matvec path -- gather, P2M, M2M, M2L, L2L, L2P, near field, scatter --
 * counted on the host as they are enqueued),
 * "tuning" (double[4]: M2L item work cap, one row per narrow box (1/0), and
 * with LFMM_AUTOTUNE the milliseconds of one FP64 M2L with the default and the
 * chosen schedule, else 0, 0),
 * "p_level" (int32[D+1]), "vfree_ptr"/"vfree_idx", "ufree_ptr"/"ufree_idx",
 * "vreact_ptr"/"vreact_idx"/"vreact_comp", "ureact_ptr"/"ureact_idx"/"ureact_comp"
 * (CSR over boxes), "components" (int32[4*ncomp]: ls, a, lt, b).
 */
lfmm_status lfmm_geometry_query(lfmm_geometry g, const char *name, void *host_out,
                                int64_t nbytes, int64_t *needed);

const char *lfmm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LFMM_H */
