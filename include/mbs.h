/*
 * mbs.h - C ABI of the GB300 modified Born series (MBS) Helmholtz solver with
 * block domain decomposition (Mache & Vellekoop, "Domain decomposition of the
 * modified Born series approach for large-scale wave propagation simulations").
 *
 * Problem (Sec. 2, Eq. helmholtz and Eq. LV): (laplacian + k^2) psi = -S on a
 * regular 3-D grid, k(r) = 2 pi n(r) / lambda, rescaled as A x = y with
 * A = c (laplacian + k^2), x = psi, y = -c S. A is split as L + V where L is the
 * angular-spectrum convolution c F^-1(k0^2 - |p|^2) F taken separately on every
 * subdomain (Sec. 3, Eq. LV_block) and V holds the scattering potential
 * c (k^2 - k0^2) plus the truncated t x t wrap-removal and transfer blocks of the
 * subdomain edges (Sec. 3, Figs. 4-5; Sec. 3.1 steps 1-5). The solve is the
 * preconditioned Richardson iteration of Eq. wavesim_iter with the scale c of
 * Eq. c_scale2 and relaxation alpha (0.75, Eq. c_scale).
 *
 * Conventions
 *  - Arrays are complex64 (interleaved float real, imaginary), C order, shape
 *    (n0, n1, n2); axis 0 is the slowest (the paper's x axis).
 *  - Pointers may be device pointers or host pointers; the library inspects
 *    each pointer (cudaPointerGetAttributes) and copies host data through the
 *    plan's stream. Host copies are counted in the timing of the call.
 *  - Every call is synchronous with respect to the host unless stated, and all
 *    device work runs on the plan's stream. Device inputs are read on that
 *    stream: work on them queued on other streams must be complete (or ordered
 *    before it) when the call is made.
 *    (The Python binding synchronises torch's current stream before each call.)
 *  - Errors are returned as mbs_status; nothing is thrown or aborted across the
 *    ABI. mbs_last_error() returns a thread-local description of the last error.
 *  - Ownership: the caller owns every array passed in; the plan copies what it
 *    needs and owns its device buffers (or the caller-provided workspace).
 *  - There is no CPU fallback: without a CUDA device every compute call fails
 *    with MBS_ECUDA.
 */
#ifndef MBS_GB300_H
#define MBS_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MBS_API __attribute__((visibility("default")))
#else
#define MBS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mbs_plan mbs_plan;

typedef enum mbs_status {
  MBS_OK = 0,
  MBS_EINVAL = 1,      /* bad argument (shape, split, t, sizes, NaN in n, ...) */
  MBS_ENOMEM = 2,      /* device memory insufficient (checked before allocating) */
  MBS_ECUDA = 3,       /* CUDA runtime error or no device */
  MBS_ENOCONV = 4,     /* max_iter reached before tol; out holds the last iterate */
  MBS_ENAN = 5,        /* residual became NaN or Inf */
  MBS_EDIVERGE = 6,    /* residual kept rising (the iteration is monotone in exact arithmetic, Sec. 2) */
  MBS_ETIMEOUT = 7,    /* a bounded device wait expired */
  MBS_EUNSUPPORTED = 8 /* size outside the supported FFT lengths or limits below */
} mbs_status;

/* Operators for mbs_apply_operator (all act on the whole decomposed grid). */
typedef enum mbs_operator {
  MBS_OP_A = 0,         /* (L + V) x: the decomposed, truncated operator (Eq. LV_block)         */
  MBS_OP_PRECOND = 1,   /* Gamma^-1 (y - A x), Gamma^-1 = (I - V)(L + I)^-1, y = -c S of the last
                           mbs_set_source (zero if none) (Sec. 2, Eq. richardson)               */
  MBS_OP_V = 2,         /* V x = c (k^2 - k0^2) x + E x (Sec. 3.1 steps 1-5)                     */
  MBS_OP_L = 3,         /* L x = c F^-1 (k0^2 - |p|^2) F x per subdomain (Eq. L-convolution)     */
  MBS_OP_PROPAGATE = 4, /* (L + I)^-1 x per subdomain                                            */
  MBS_OP_E = 5,         /* E x: the edge-correction part of V alone                              */
  MBS_OP_FFT = 6,       /* unnormalised forward DFT of every subdomain, in place of the subdomain */
  MBS_OP_IFFT = 7       /* inverse DFT (1/n0 n1 n2) of every subdomain                           */
} mbs_operator;

/* Limits of the library. */
#define MBS_MAX_SPLIT 16 /* subdomains per axis */
#define MBS_MAX_T 40     /* truncation width (Fig. 7 sweeps t = 0..40): every t in 1..40; widths
                            1..16, 20, 24 and 32 have specialised correction kernels, the others a
                            generic one (the tensor-core form takes t <= 32) */
#define MBS_T_NONE (-1)  /* mbs_options.truncation value for t = 0: no edge corrections at all
                            (uncoupled periodic subdomains; the t = 0 end of Fig. 7)        */
#define MBS_MAX_EDGE 512 /* longest subdomain edge. Edges <= 512 whose prime factors are 2, 3,
                            5 and 7 have mixed-radix FFT kernels (106 lengths); any other edge
                            <= 256 is transformed by Bluestein's algorithm on one of them */

/* Option flags. */
#define MBS_FLAG_NO_GRAPH (1u << 0)  /* launch kernels one by one instead of replaying a CUDA graph */
#define MBS_FLAG_CORR_TF32 (1u << 1) /* edge-correction contractions on the tensor cores as 3xTF32 with
                                        FP32 accumulation (mma.sync m16n8k8): the separate correction
                                        launches (axes 0 and 1 in the iteration, all axes in the
                                        operators); the axis-2 terms the iteration fuses into its
                                        first pass and layer update stay FP32. Needs every corrected
                                        subdomain edge >= 2t. Default: FP32 CUDA-core products.   */
#define MBS_FLAG_RESIDUAL_FORM (1u << 2) /* iterate on r'_n = Gamma^-1 (A x_n - y) instead of x_n:
                                        r'_{n+1} = r'_n - alpha Gamma^-1 A r'_n, x_{n+1} = x_n - alpha r'_n
                                        (compensated sum). The same iterates as Eq. wavesim_iter in exact
                                        arithmetic; in complex64 the residual has no floor set by ||x||,
                                        so tolerances below that floor are reachable. Costs about
                                        24 B per voxel and iteration more (x and its low word).      */
#define MBS_FLAG_NO_TMA (1u << 3) /* feed the axis-1 FFT passes with per-thread global loads instead
                                     of tensor-map (TMA) copies into double-buffered shared memory.
                                     Default: TMA where the edge has TMA kernels (32, 64, 128, 256,
                                     320), the grid's row pitch is a multiple of 16 bytes and the
                                     plan-time timing finds TMA faster.                           */
#define MBS_FLAG_FORCE_TMA (1u << 4) /* keep every tensor-map feed the plan can build, without the
                                     plan-time timing, and feed the axis-0 pass (forward transform,
                                     propagator, inverse) by TMA too, which only this flag does
                                     (results are identical)                                      */
#define MBS_FLAG_PLAIN_STEPS (1u << 5) /* comparison form of the iteration: every step of
                                     Eq. wavesim_iter is its own launch over the whole grid (E x,
                                     u = B x + y - E x, three forward FFT passes, the propagator,
                                     three inverse passes, d = x - w, E d, r = B d - E d, |r|^2,
                                     the update), no fused prologues or epilogues, no CUDA graph,
                                     and the residual summed and the stop test taken on the host
                                     after every iteration. Same iterates as the default form up to
                                     FP32 rounding; not with MBS_FLAG_RESIDUAL_FORM or in batches. */
#define MBS_FLAG_ACTIVATION (1u << 6) /* subdomain activation (Sec. 3.1, "Implementation"): after
                                     mbs_set_source only the subdomains that meet the bounding box of
                                     the source's non-zero voxels are computed; every graph_iters
                                     iterations an inactive subdomain next to an active one is
                                     activated once the norm of the field that neighbour transfers
                                     into its boundary layers exceeds activation_threshold *
                                     ||r_0||. The inactive subdomains keep x = 0 and add nothing to
                                     the residual, so the early iterates differ slightly from the
                                     unmasked ones; the iteration converges to the same solution
                                     (it converges from any start). mbs_iterate polls the device
                                     between replays while any subdomain is inactive, no_poll or
                                     not. The default (x) form only; needs t > 0, mixed-radix axis-2
                                     edges and 2 t S_2 <= 64; not in batches. A warm start
                                     (mbs_set_initial_field) activates every subdomain.          */
#define MBS_FLAG_NO_TUNE (1u << 7) /* skip the plan-time tuner (see mbs_plan_info.tuning) and its
                                     on-disk cache: TMA feed wherever a tensor map exists, with as
                                     many CTAs per SM as fit, and side-split correction kernels of
                                     128 threads. The tuner only chooses launch shapes, so tuned and
                                     untuned plans give bit-identical iterates. The cache file is
                                     MBS_TUNE_CACHE if that environment variable is set (empty: no
                                     cache), else $XDG_CACHE_HOME (or $HOME/.cache) /mbs_gb300/
                                     tune-v1.txt, one line per (device, SM count, build, pass, edge,
                                     grid) key.                                                   */

typedef struct mbs_options {
  int32_t truncation;        /* t, the kept edge width (Sec. 3, Fig. 5); 0 -> 8 (Sec. 3.3);
                                MBS_T_NONE -> t = 0                                              */
  double alpha;              /* relaxation (Eq. c_scale); 0 -> 0.75                              */
  uint32_t periodic_mask;    /* bit d set: axis d periodic. Periodic unsplit axis: no corrections
                                (a_d = 0); periodic split axis: transfer across the seam (a_d = 2) */
  double absorb_kappa;       /* peak imaginary index of the absorbing ramps; <0 -> 0.5           */
  const int64_t *split_sizes;/* NULL (near-equal sizes, the first n mod S one larger) or
                                split[0]+split[1]+split[2] explicit sizes, axis by axis           */
  uint32_t flags;            /* MBS_FLAG_*                                                        */
  int32_t graph_iters;       /* iterations per captured graph; 0 -> chosen by the plan            */
  void *stream;              /* cudaStream_t for all work; NULL -> a non-blocking stream the plan creates */
  void *workspace;           /* optional device workspace of workspace_bytes (see
                                mbs_workspace_bytes); NULL -> the plan allocates its own          */
  size_t workspace_bytes;
  int64_t tma_wait_cycles;   /* bound of each wait for a tensor-map copy in the iteration and the
                                operators, in SM clock cycles; 0 -> about 2 s. Past it the call
                                returns MBS_ETIMEOUT (a short bound lets a test provoke that path
                                with copies that do complete)                                     */
  double activation_threshold; /* MBS_FLAG_ACTIVATION: relative norm of the transferred field
                                that activates a subdomain; 0 -> 1e-3                             */
} mbs_options;

/* Fill *opts with the defaults above. */
MBS_API void mbs_default_options(mbs_options *opts);

/*
 * Create a plan: the problem of Sec. 2 on a grid `shape` (n0, n1, n2) with pixel
 * size `pixel_size` and vacuum wavelength `wavelength` (same length unit),
 * refractive index `refractive_index` (complex64, shape; host or device), and
 * absorbing layers of boundary_widths[2d], boundary_widths[2d+1] pixels on the
 * low and high face of axis d (added inside the grid as a linear ramp of the
 * imaginary index, absorb_kappa * (w - i)/w at depth i from a face of width w;
 * where faces meet the largest ramp applies). `split` gives the subdomains per axis (Sec. 3: any number
 * along any axis, unequal sizes allowed). The plan computes, in FP64 on the
 * device: k^2, k0^2 (centre of the bounding box of k^2 in C), the scale c of
 * Eq. c_scale2 with ||A12|| the spectral norm of the t x t block W, and the
 * medium factor B = 1 - c (k^2 - k0^2) stored as complex64.
 * Errors: MBS_EINVAL (shape < 1, split not in [1, MBS_MAX_SPLIT], t < 0 or
 * > MBS_MAX_T, t larger than a subdomain edge on a corrected axis, non-finite n,
 * wavelength or pixel size <= 0), MBS_EUNSUPPORTED (an edge outside the FFT
 * lengths of MBS_MAX_EDGE), MBS_ENOMEM (buffers do not fit; nothing is allocated), MBS_ECUDA.
 */
MBS_API mbs_status mbs_plan_create(mbs_plan **plan, const int64_t shape[3], double pixel_size, double wavelength,
                           const void *refractive_index, const int32_t boundary_widths[6],
                           const int32_t split[3], const mbs_options *opts);

/* Device bytes a plan with these arguments needs (for a caller-provided workspace). */
MBS_API mbs_status mbs_workspace_bytes(const int64_t shape[3], const int32_t split[3], const mbs_options *opts,
                               size_t *bytes);

typedef struct mbs_plan_info {
  double c_re, c_im;         /* scale factor c (Eq. c_scale2)                                  */
  double k0sq_re, k0sq_im;   /* background k0^2                                                */
  double contrast;           /* ||k^2 - k0^2||_inf                                             */
  double block_norm;         /* ||W||_2 in units of 1/h^2 (R2 reading of ||A12||)              */
  int32_t a[3];              /* a_d of Eq. c_scale2                                            */
  int32_t t;
  double alpha;
  int64_t shape[3];
  int32_t split[3];
  int64_t sizes[3][MBS_MAX_SPLIT];  /* subdomain edges along each axis                        */
  size_t device_bytes;       /* device memory held by the plan                                 */
  int32_t graph_iters;
  int32_t tma_groups;        /* edge groups whose axis-1 pass (or, with MBS_FLAG_FORCE_TMA, axis-0
                                pass) is fed by TMA (chosen at plan creation by timing both feeds;
                                results are identical)                                          */
  int32_t tune_source;       /* launch shapes: 0 defaults (MBS_FLAG_NO_TUNE, MBS_FLAG_FORCE_TMA or
                                nothing to tune), 1 timed at plan creation, 2 from the cache     */
  char tuning[256];          /* the choices, e.g. "axis1/320:tmax1 corr01:side/128" (axis-1 pass
                                of edge 320 TMA-fed with one CTA per SM)                        */
} mbs_plan_info;

MBS_API mbs_status mbs_plan_get_info(const mbs_plan *plan, mbs_plan_info *info);

/*
 * out = op(x) for op in mbs_operator. x and out are complex64 arrays of the
 * grid's shape (host or device); they must not alias. MBS_OP_FFT / MBS_OP_IFFT
 * return every subdomain's transform in the subdomain's own box, k-space index
 * in natural (FFT) order.
 */
MBS_API mbs_status mbs_apply_operator(mbs_plan *plan, int32_t which, const void *x, void *out);

/*
 * Start a solve: store the source S (complex64, shape; host or device; copied
 * into the plan), set x = 0 and clear the residual history. The iteration uses
 * y = -c S (Eq. LV); only the bounding box of S's non-zeros is read per step.
 */
MBS_API mbs_status mbs_set_source(mbs_plan *plan, const void *source);

/*
 * Warm start (resume): after mbs_set_source, replace the field x = 0 by x0
 * (complex64, shape; host or device) and restart the iteration count and the
 * history. The iteration converges from any start (Sec. 3.1); eps_n stays
 * normalised by ||Gamma^-1 y||, the residual of x = 0, so a solve resumed from
 * its last field continues with the same eps (eps_0 < 1 for a good x0).
 * Uses (and on first use allocates) the plan's staging buffers. Errors:
 * MBS_EINVAL without a source.
 */
MBS_API mbs_status mbs_set_initial_field(mbs_plan *plan, const void *x0);

/*
 * Run up to n_iter iterations of Eq. wavesim_iter from the current state,
 * stopping after the update in which eps_n = ||r_n|| / ||r_0|| < tol (Sec. 3.1;
 * r_n = Gamma^-1 (y - A x_n) is taken before update n, x_0 = 0, FP64 norms).
 * *iters_done (nullable) receives the total iterations since mbs_set_source,
 * *residual (nullable) the last eps. Returns MBS_OK if eps < tol was reached,
 * MBS_ENOCONV if the budget ran out, MBS_ENAN / MBS_EDIVERGE on breakdown.
 * If `no_poll` is non-zero the call enqueues all n_iter iterations without
 * intermediate host synchronisation (for timing); it still synchronises once
 * at the end.
 */
MBS_API mbs_status mbs_iterate(mbs_plan *plan, int32_t n_iter, double tol, int32_t no_poll, int32_t *iters_done,
                       double *residual);

/*
 * Subdomain activation state (MBS_FLAG_ACTIVATION): flags[s] = 1 if subdomain s
 * is computed, s = (j0 * split[1] + j1) * split[2] + j2, for s < cap (flags
 * nullable); *n_active (nullable) receives the number of active subdomains.
 * Without the flag every subdomain is active.
 */
MBS_API mbs_status mbs_get_active_subdomains(const mbs_plan *plan, int32_t *flags, int32_t cap, int32_t *n_active);

/* Copy the current field x (complex64, shape) to out (host or device). */
MBS_API mbs_status mbs_get_field(const mbs_plan *plan, void *out);

/*
 * Copy the residual history eps_0 .. eps_{n-1} (n = min(cap, iterations done))
 * to host memory `history`; *n_out receives n.
 */
MBS_API mbs_status mbs_get_history(const mbs_plan *plan, double *history, int32_t cap, int32_t *n_out);

/*
 * Full solve: mbs_set_source(source), mbs_iterate(max_iter, tol), then the
 * field to `out` (host or device; may alias `source`). `history` (nullable,
 * host) receives up to max_iter residuals. Returns as mbs_iterate; on
 * MBS_ENOCONV `out` holds the last iterate.
 */
MBS_API mbs_status mbs_solve(mbs_plan *plan, const void *source, void *out, double tol, int32_t max_iter,
                     int32_t *iters_out, double *residual_out, double *history);

/*
 * Timing support: run n_iter iterations (tol 0) launching kernels one by one
 * with CUDA events around every launch on the plan's stream, and report per
 * kernel kind the number of launches and the summed device milliseconds.
 * kind names: mbs_kernel_kind_name(i) for i < MBS_KERNEL_KINDS.
 */
#define MBS_KERNEL_KINDS 8
MBS_API mbs_status mbs_profile_iterations(mbs_plan *plan, int32_t n_iter, int32_t launches[MBS_KERNEL_KINDS],
                                  double ms[MBS_KERNEL_KINDS]);
MBS_API const char *mbs_kernel_kind_name(int32_t kind);

/*
 * Edge corrections without allocation: out = E x, the same operator as
 * mbs_apply_operator(plan, MBS_OP_E, x, out) (the paper has no counterpart of
 * this entry point). It is for callers that must not trigger a device
 * allocation when they call, for instance a process whose device memory is
 * handed out entirely by another framework's caching allocator or by a fixed
 * memory budget: mbs_apply_operator may allocate staging buffers on first use.
 * Here the correction scratch is a fixed 16 MiB array inside the library (every
 * GPU that loads the library holds it until the process exits), the plan's own
 * buffers are not touched, and the call allocates nothing.
 *  - x and out: device pointers on the plan's device only (complex64, the plan's
 *    grid); host pointers are rejected with MBS_EINVAL because they would need a
 *    staging buffer, and so are pointers on another device. The plan's device
 *    must be current.
 *  - grids above 2^21 voxels (the scratch's capacity) are rejected with MBS_EINVAL.
 *  - The scratch's device address is looked up once per device, with that
 *    device current: mbs_plan_create does it for the plan's device (loading the
 *    library's module that holds the array); if that failed, the first call here
 *    does it and should then come before any stream capture.
 *  - All calls share the scratch: calls whose work overlaps on the GPU (on
 *    different streams or plans) race. The work runs on the plan's stream and the
 *    call synchronises that stream before it returns.
 *  - Errors: mbs_noalloc_last_error() describes the last failure of this call.
 */
MBS_API mbs_status mbs_apply_edge_corrections_noalloc(const mbs_plan *plan, const void *x, void *out);
MBS_API const char *mbs_noalloc_last_error(void);

/*
 * Batches of independent solves (e.g. the frequencies of a transient
 * simulation, which the paper solves one by one, Sec. 1), advanced together:
 * one CUDA graph holds graph_iters iterations of every plan, each plan on its
 * own stream forked from the batch stream so the solves run concurrently. Every
 * plan keeps its own source (mbs_set_source), state, stop test and history; a
 * converged plan's kernels leave at once. Plans must live on the current device
 * and must not be iterated elsewhere while the batch runs. stream: NULL -> a
 * stream the batch creates. graph_iters: 0 -> 10.
 */
typedef struct mbs_batch mbs_batch;
MBS_API mbs_status mbs_batch_create(mbs_batch **batch, int32_t nplans, mbs_plan *const *plans, void *stream,
                                    int32_t graph_iters);
/*
 * Run up to n_iter iterations of every plan (as mbs_iterate); per plan
 * (nullable arrays of nplans entries): total iterations, last residual, status
 * (MBS_OK reached tol, MBS_ENOCONV, MBS_ENAN, MBS_EDIVERGE). Returns MBS_OK if
 * every plan reached tol, MBS_ENOCONV if some did not, or the first error.
 */
MBS_API mbs_status mbs_batch_iterate(mbs_batch *batch, int32_t n_iter, double tol, int32_t no_poll, int32_t *iters,
                                     double *residuals, int32_t *statuses);
/*
 * Kernel launches per iteration of the whole batch (-1 on error); *fused
 * (nullable) is 1 when the batch runs in its fused form: plans that share a
 * subdomain edge along some axis form a cluster, and each cluster takes one
 * launch per pass and subdomain edge over its plans (grid.z or grid.y selecting
 * the plan); the clusters run side by side on streams of the batch. The form
 * applies when every plan iterates in the default x form with FP32
 * corrections, every subdomain edge is a mixed-radix length of at most 128
 * (and at least 2t on corrected axes 0 and 1) and all plans share t; otherwise
 * the batch graph holds every plan's own launches.
 */
MBS_API int32_t mbs_batch_launches_per_iteration(mbs_batch *batch, int32_t *fused);
/*
 * Choose the batch's form: on = 1 the fused form (MBS_EINVAL if the plans do
 * not allow it), 0 the graph of every plan's own launches. mbs_batch_create
 * picks the fused form whenever the plans allow it. Iterates are the same in
 * both forms.
 */
MBS_API mbs_status mbs_batch_set_fused(mbs_batch *batch, int32_t on);
MBS_API void mbs_batch_destroy(mbs_batch *batch);

MBS_API void mbs_plan_destroy(mbs_plan *plan);

/*
 * 1 if this library was built with MBS_BOUNDS_CHECK: every kernel then checks
 * the index range of its accesses to the grid arrays, skips an access outside
 * the grid (nothing traps) and counts it in error words of the plan, and
 * mbs_iterate, mbs_apply_operator and mbs_batch_iterate return MBS_EINVAL with
 * the first offending site, index and limit in mbs_last_error(). 0 for the
 * normal build, where the checks compile away.
 */
MBS_API int32_t mbs_build_checks_bounds(void);

/* Thread-local description of the last error (empty string if none). */
MBS_API const char *mbs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MBS_GB300_H */
