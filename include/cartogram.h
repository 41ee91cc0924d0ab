/*
 * cartogram.h - C-ABI of the GB300 (sm_103a) diffusion-flow cartogram library.
 *
 * The library computes density-equalising map projections (cartograms) with the
 * flow-based method of Gastner, Seguy & More, "Fast flow-based algorithm for
 * creating density-equalizing map projections" (PNAS 2018, arXiv:1802.07625),
 * integrating the diffusion flow (SI Appendix section 2, Eq. fmn_diff): the cosine
 * spectrum of the blurred, rasterised density is damped in time, inverse cosine /
 * sine transforms give rho and grad rho, v = -grad(rho)/rho, and all Lx*Ly grid
 * points advance by an adaptive predictor-corrector step with bilinear
 * interpolation (main text, section "Flow-based cartograms" and the paragraph on
 * overlaying an Lx x Ly grid). Polygon vertices follow through the projected grid,
 * and the integration repeats on its own output until every region's area is
 * within the tolerance of its target (main text, section on benchmarking).
 *
 * Coordinates are grid units inside the box [0, Lx] x [0, Ly]. Grid points are the
 * cell centres (i + 1/2, j + 1/2). Fields are row-major Lx*Ly arrays indexed
 * [j*Lx + i]; spectra are indexed [n*Lx + m] (m: x wavenumber).
 *
 * Pointers: every array argument may be host memory or device memory of the
 * context's GPU; the library detects which and copies accordingly. The caller owns
 * every buffer it passes; the library copies inputs during the call and never keeps
 * a caller pointer. All functions are synchronous with respect to the host unless
 * stated otherwise; device work runs on the context's stream, which does not wait for
 * other streams: device inputs produced on another stream must be complete (or that
 * stream passed to cartogram_set_stream) before the call.
 *
 * Errors: functions return CG_OK (0) or a negative CG_E* code; a description of
 * the last error is available from cartogram_last_error(). A context is not thread
 * safe: use one context per host thread.
 */
#ifndef CARTOGRAM_H
#define CARTOGRAM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cg_ctx cg_ctx;

enum {
    CG_OK = 0,
    CG_EINVAL = -1,        /* invalid argument (sizes, NaN/Inf, non-positive value, ...) */
    CG_ENOMEM = -2,        /* device or host allocation failed */
    CG_ECUDA = -3,         /* a CUDA runtime call failed */
    CG_ENOCONVERGE = -4,   /* max_iter outer iterations did not reach area_tol */
    CG_EFOLD = -5,         /* a projected grid folded over (non-positive quad area) */
    CG_ESTEPFAIL = -6,     /* an integration used max_steps attempts, or its step collapsed */
    CG_ETIMEOUT = -7,      /* the call's time_limit passed, or a bounded device-side wait
                              (grid barrier, bulk copy) gave up */
    CG_ESTATE = -8         /* call out of order (e.g. integrate before set_regions) */
};

enum {
    CG_PRECISION_FP64 = 0,   /* every field, transform and position in FP64 */
    CG_PRECISION_MIXED = 1,  /* inverse transforms, fields and displacements in FP32; the
                                forward transform in float-float arithmetic (about 48 bits,
                                FP64 input and spectrum); rasterisation, polygon areas, the
                                convergence test and the step-control arithmetic in FP64 */
    CG_PRECISION_MIXED_FF = 2 /* as CG_PRECISION_MIXED, with the second inverse transform pass
                                (the column transforms that form rho, grad rho and v) in
                                float-float arithmetic (about 48 bits on FP32 hardware): FP32
                                rounding at the scale of a column's largest densities no longer
                                swamps regions far below them. Not for use_graph = 2 (runs as 1) */
};

enum {
    CG_FLOW_DIFFUSION = 0,   /* diffusion flow, SI Eq. fmn_diff: the density at time t comes
                                from the damped spectrum, two transform passes per step */
    CG_FLOW_LINEAR = 1       /* linear equalisation, SI Eq. fmn_fast (the paper's method):
                                rho(t) = (1 - t) rho0 + t rho_bar, a flux J = -grad Phi that is
                                constant in time (SI Eqs. Jxmn, Jymn), integration to t = 1 */
};

/* Tuning of the method. cartogram_default_options() fills the defaults noted here. */
typedef struct cg_options {
    int precision;      /* CG_PRECISION_FP64 (default), CG_PRECISION_MIXED or CG_PRECISION_MIXED_FF */
    double dt0;         /* first trial step, diffusion time with D = 1 (1e-2) */
    double atol;        /* accept a step when max ||r_corr - r_pred|| <= atol cells (1e-2) */
    double grow;        /* step factor after an accepted step (1.2) */
    double shrink;      /* step factor after a rejected step (0.5) */
    double cfl;         /* step cap: h * max|v| <= cfl cells (1.0) */
    double rho_tol;     /* an integration ends at the first accepted step with
                           max |rho - rho_bar| / rho_bar <= rho_tol (1e-4) */
    double area_tol;    /* outer iterations end when max |A_i/A^_i - 1| < area_tol (0.01) */
    int max_steps;      /* attempted steps per integration before CG_ESTEPFAIL (4000) */
    int max_iter;       /* outer iterations before CG_ENOCONVERGE (500). Regions whose target
                           is about one cell wide shrink by a few percent per iteration once
                           the grid stops resolving them: the 512^2 clustered map with
                           lognormal(1.5) values needs about 190 */
    int use_graph;      /* how an integration's step loop runs: 1 (default) one CUDA-graph
                           launch whose conditional WHILE node repeats the per-phase kernels;
                           2 one persistent cooperative kernel whose phases meet at grid
                           barriers (falls back to 1 where a cooperative launch does not fit);
                           0 the same per-phase kernels launched by a host loop */
    double blur_decay;  /* blur width of outer iteration k (counted from set_regions/reset) is
                           blur_width * blur_decay^k (0.5); 1: the same blur in every
                           iteration, 0: only the first integration is blurred */
    int autotune;       /* 1: time the candidate launch shapes of the step kernels on first
                           use and keep the fastest (default); 0: heuristic shapes */
    int flow;           /* CG_FLOW_DIFFUSION (default) or CG_FLOW_LINEAR. With the linear flow
                           dt0 is in units of its time t in [0, 1], every integration ends at
                           t = 1, rho_tol is not used, and use_graph = 2 runs as 1 */
    double time_limit;  /* seconds of device time one cartogram_integrate (or one batch call,
                           per context) may take; 0 (default): no limit. The device clock is
                           read when the call starts and by the step controller after every
                           attempted step: past the limit, the integration in flight ends with
                           CG_ETIMEOUT and maps nothing (the vertices and history keep the
                           iterations completed before it). Must be finite and >= 0 */
    long long barrier_spins; /* use_graph = 2: polls of one grid-barrier wait before the
                           persistent kernel gives up and the integration ends with
                           CG_ETIMEOUT, mapping nothing (2^25, about a second); from 1 to
                           2^40 */
} cg_options;

typedef struct cg_stats {
    int iterations;             /* outer iterations run by the last cartogram_integrate */
    int converged;              /* 1 if max area error < area_tol */
    long long steps_accepted;   /* summed over the iterations */
    long long steps_rejected;
    double max_area_error;      /* max_i |A_i / A^_i - 1| after the last iteration */
    double t_end;               /* diffusion time reached by the last integration */
    double seconds;             /* host wall time of the call */
    double step_loop_ms;        /* device time of the integrations' step loops */
} cg_stats;

/* Fill *opt with the defaults listed in cg_options. Returns CG_OK or CG_EINVAL (NULL). */
int cartogram_default_options(cg_options* opt);

/* Create a context for an Lx x Ly grid (main text: "overlay the map with an Lx x Ly
 * square grid"; Lx and Ly integers). This build supports powers of two from 8 to
 * 1024 along each axis. blur_width is the standard deviation, in cells, of the
 * Gaussian blur applied to the rasterised density before every integration (main
 * text, section on benchmarking: "Gaussian blur of moderate width"); 0 disables
 * it. opt may be NULL for the defaults. Allocates the device state on the current
 * CUDA device. On success *out owns the context; free it with cartogram_destroy.
 * Errors: CG_EINVAL (sizes, blur, options), CG_ENOMEM, CG_ECUDA. */
int cartogram_init(int Lx, int Ly, double blur_width, const cg_options* opt, cg_ctx** out);

/* Run the context's device work on `cuda_stream` (a cudaStream_t, e.g. torch's current
 * stream) from now on; NULL selects the context's own stream. */
int cartogram_set_stream(cg_ctx* ctx, void* cuda_stream);

/* Set the map: n_regions regions with target values (main text, problem statement:
 * areas proportional to e.g. population; the density of a region is its value over
 * its area, section on previous all-coordinates methods).
 *   target_values [n_regions]      > 0 and finite
 *   ring_offsets  [n_rings + 1]    int64, ring k owns vertices ring_offsets[k] ..
 *                                  ring_offsets[k+1]-1; ring_offsets[0] = 0, increasing,
 *                                  at least 3 vertices per ring
 *   ring_region   [n_rings]        int32 in [0, n_regions)
 *   xy            [ring_offsets[n_rings]][2]  vertices (x, y) inside [0,Lx]x[0,Ly];
 *                                  rings are implicitly closed; counter-clockwise rings
 *                                  are outer boundaries, clockwise rings are holes, and
 *                                  a region's area is the signed sum over its rings.
 * Regions must not overlap and each must have positive area. Resets the iteration
 * history. A map with the same ring_offsets and ring_region as the current one (new values
 * or moved vertices, e.g. the frames of an animation) reuses the context's device buffers
 * and captured graphs. Errors: CG_EINVAL, CG_ENOMEM, CG_ECUDA. */
int cartogram_set_regions(cg_ctx* ctx, int n_regions, const double* target_values,
                          int64_t n_rings, const int64_t* ring_offsets,
                          const int32_t* ring_region, const double* xy);

/* Run the whole method (main text, section on benchmarking, "repeat the integration"):
 * rasterise, blur and transform the density, integrate the flow of all grid points
 * to equalisation, map the vertices through the projected grid, recompute the areas,
 * and repeat until max_i |A_i/A^_i - 1| < area_tol (main text: a maximum relative
 * area error below 1%), where A^_i = V_i * sum(A) / sum(V). Continues from the
 * current vertices, so a second call after convergence runs no iteration. stats may
 * be NULL. Returns CG_OK on convergence, CG_ENOCONVERGE after max_iter iterations
 * (the vertices and history stay valid), CG_ESTEPFAIL, CG_ESTATE, CG_ECUDA.
 * With use_graph = 1 the whole outer iteration runs on the device: one CUDA-graph
 * launch whose conditional WHILE node repeats rasterisation, transform, integration
 * (itself a WHILE node), mapping and areas until the areas converge; the host reads
 * the outcome once (the first call first runs one iteration from the host when the
 * launch shapes are still to be tuned, and a launch that runs out of history slots
 * is repeated after more are allocated). use_graph = 0 or 2 run the outer loop from
 * the host, reading the outcome after every integration. */
int cartogram_integrate(cg_ctx* ctx, cg_stats* stats);

/* Map n arbitrary points (x, y pairs, [n][2]) through every projected grid of the
 * history in order (main text: the projection is defined for every point, e.g. the
 * capitals or death cases of the case studies). xy_in and xy_out may alias. Errors:
 * CG_EINVAL, CG_ECUDA. */
int cartogram_project(cg_ctx* ctx, int64_t n, const double* xy_in, double* xy_out);

/* Preimages under the composed projection (the main text's inverse graticule: features
 * found on the cartogram identified in the original domain): every projected grid of the
 * history inverted in reverse order. Each grid's map is the bilinear map that
 * cartogram_project applies (the quads along the walls extended to the box edge); its
 * inverse is found by Newton's method inside a quad, walking to the neighbouring quad
 * until the solution lies in the current one. cartogram_inverse_project(project(p)) = p
 * wherever the grids do not fold. Points without a preimage in the box (outside it, or
 * where a walk does not settle) come back as NaN. xy_in and xy_out may alias and may be
 * host or device memory. Errors: CG_EINVAL, CG_ECUDA. */
int cartogram_inverse_project(cg_ctx* ctx, int64_t n, const double* xy_in, double* xy_out);

/* Angular distortion of the composed projection (SI section 3, the Tissot indicatrix):
 * at the centre of every quad of the original cell-centre lattice ((Lx-1)(Ly-1) points),
 * the Jacobian of the composed bilinear maps by the chain rule, its singular values
 * a >= b, e = ln(a/b) and e~ = 2 asin((a - b)/(a + b)). out[4] = {e_a, e_inf, e~_a,
 * e~_inf}: the means and maxima over those points (SI: the average and the supremum
 * over the Lx x Ly box). An empty history (the identity) gives zeros. FP64 on the
 * stored displacements. Errors: CG_EINVAL, CG_ECUDA. */
int cartogram_distortion(cg_ctx* ctx, double* out);

/* Loss of `iterations` outer iterations and its gradient with respect to the regions'
 * target values and the blur width (reverse mode through the whole method: region areas
 * and weights, rasterisation (the exact coverage, also as a function of the vertices
 * entering each later iteration), blurred forward transform, every predictor-corrector step
 * with its interpolations and transforms, the vertex maps and the areas). From the current
 * vertices X (left unchanged; no history entry is added) with target values
 * V = values[n_regions] and blur width blur_width (iteration k blurs with
 * blur_width * blur_decay^(h + k), h = history length, as cartogram_integrate does):
 * X' = X carried through the iterations, A' its region areas, A^_i = V_i sum(A') / sum(V),
 *   loss = sum_i (ln A'_i - ln A^_i)^2 + lambda * sum_v |X'_v - X_v|^2.
 * Each integration's accepted steps form a schedule: replay = 0 integrates adaptively (with
 * these values) and records the schedules; replay = 1 reuses the last recorded ones (same
 * number of iterations, steps and sizes), so that the loss is a smooth function of
 * (values, blur_width), e.g. for finite differences. Positions are stored every `checkpoint`
 * steps (>= 1) and recomputed in between on the way back. loss, grad_values[n_regions] and
 * grad_blur may each be NULL (with both gradients NULL only the forward runs). Needs the
 * FP64 path and the diffusion flow. Errors: CG_EINVAL, CG_ESTATE (no map; replay without a
 * recorded schedule of as many iterations), CG_ESTEPFAIL, CG_EFOLD (a mapped region with
 * non-positive area), CG_ENOMEM, CG_ECUDA. */
int cartogram_iteration_gradient(cg_ctx* ctx, const double* values, double blur_width, double lambda, int iterations,
                                 int replay, int checkpoint, double* loss, double* grad_values, double* grad_blur);

/* Vector-Jacobian product of `iterations` outer iterations, for a loss of the caller's
 * choosing on the mapped vertices and areas (the reverse mode of
 * cartogram_iteration_gradient with the loss left to the caller). From the current
 * vertices X (left unchanged; no history entry is added) with target values
 * V = values[n_regions] and blur width blur_width, the iterations give the mapped vertices
 * X' and their region areas A' (SI Eq. det: the areas the cartogram equalises).
 *   xy_out     [n_vertices][2] FP64: X' (may be NULL)
 *   area_out   [n_regions] FP64: A' (may be NULL)
 *   grad_xy    [n_vertices][2] FP64: dL/dX' of the caller's loss (NULL: zero)
 *   grad_area  [n_regions] FP64: dL/dA' (NULL: zero)
 *   grad_values[n_regions], grad_blur: receive (dX'/dV)^T dL/dX' + (dA'/dV)^T dL/dA' and the
 *              same for the blur width (each may be NULL; with both NULL only the forward
 *              runs). A term of the loss that depends on V directly is not included.
 * replay and checkpoint are as for cartogram_iteration_gradient (a forward call with
 * replay = 0 records the step schedules, a later call with replay = 1 differentiates that
 * same function). Every array may be host or device memory. Needs the FP64 path and the
 * diffusion flow. Errors: CG_EINVAL (arguments, non-finite adjoints), CG_ESTATE,
 * CG_ESTEPFAIL, CG_ENOMEM, CG_ECUDA. */
int cartogram_iteration_vjp(cg_ctx* ctx, const double* values, double blur_width, int iterations, int replay,
                            int checkpoint, double* xy_out, double* area_out, const double* grad_xy,
                            const double* grad_area, double* grad_values, double* grad_blur);

/* Signed relative area errors A_i / A^_i - 1 of the current vertices, [n_regions]. */
int cartogram_area_errors(cg_ctx* ctx, double* err);

/* Current (mapped) vertices, same layout as set_regions' xy. */
int cartogram_get_vertices(cg_ctx* ctx, double* xy_out);

/* Restore the vertices given to the last cartogram_set_regions and clear the history,
 * on the device (no host transfer). Errors: CG_ESTATE (no map). */
int cartogram_reset(cg_ctx* ctx);

/* Polygon-level distortion measures (SI section 4) of the current vertices against those given
 * to the last cartogram_set_regions (a region's points are the vertices of all its rings):
 *   out[0]  mean over the regions of the aspect ratio (longer / shorter side) of the
 *           bounding rectangle of minimum area over all orientations (exact: found along
 *           the edges of the region's convex hull; NaN for a hull of more than 2048 vertices)
 *   out[1]  relative position error theta in [0, 1]: the angle between c_i - c_j and
 *           d_i - d_j averaged over all pairs of regions and divided by pi, c the centroids
 *           on the input map and d on the current one
 *   out[2]  the mean aspect ratio of the input map's regions
 * The paper's third measure (the total Hamming distance, a minimum over translations of a
 * symmetric difference of polygons) is not computed. out: 3 doubles, host or device.
 * Errors: CG_EINVAL (NULL), CG_ESTATE (no map), CG_ECUDA. */
int cartogram_polygon_measures(cg_ctx* ctx, double* out);

/* New target values for the current map (the frames of an animation, replicates of the
 * data; main text, problem statement: areas proportional to the values): restores the
 * vertices given to the last cartogram_set_regions, clears the history and recomputes the
 * area errors, keeping every device buffer and captured graph.
 *   target_values [n_regions of the map]  > 0 and finite; host or device pointer
 * Errors: CG_EINVAL (NULL or invalid values, nothing changed), CG_ESTATE (no map), CG_ECUDA. */
int cartogram_set_values(cg_ctx* ctx, const double* target_values);

/* Number of outer iterations in the history (projected grids stored). */
int cartogram_history_length(const cg_ctx* ctx);

/* What outer iteration k of the history did (main text, section on benchmarking: the
 * integration is repeated until the largest relative area error is below 1 %): out[6] =
 * {max_i |A_i/A^_i - 1| once its vertices were mapped, diffusion time its integration
 * reached, accepted steps, rejected steps, device time of its step loop in ms, blur width it
 * used}. out may be host or device memory. Errors: CG_EINVAL (k out of range). */
int cartogram_iteration_record(cg_ctx* ctx, int k, double* out);

/* Projected grid of history entry k: positions of the Lx*Ly cell centres after
 * integration k, xy_out [Lx*Ly][2] FP64. Errors: CG_EINVAL (k out of range). */
int cartogram_get_grid(cg_ctx* ctx, int k, double* xy_out);

/* Fold check of history entry k (SI Eq. det: a density-equalising map has a positive
 * Jacobian everywhere): the signed area of every quad of neighbouring projected grid
 * points. *n_folded (may be NULL) receives the number of quads with non-positive area,
 * *min_area (may be NULL) the smallest area in cells^2. Errors: CG_EINVAL (k). */
int cartogram_fold_count(cg_ctx* ctx, int k, long long* n_folded, double* min_area);

/* ---- step-level entry points (one stage of the method each) ---------------- */

/* Rasterised density of the current vertices, normalised so that the box mean is 1
 * (section on previous all-coordinates methods; the margin carries the mean density,
 * section on benchmarking): rho[j*Lx+i] = rho0/rho_bar with exact cell coverage.
 * rho_out [Lx*Ly] FP64. */
int cartogram_density(cg_ctx* ctx, double* rho_out);

/* Cosine spectrum (main text Eq. rhotilde_mn) of the normalised density of the
 * current vertices, times the Gaussian blur factor exp(-pi^2 s^2 (m^2/Lx^2 +
 * n^2/Ly^2)/2). spec_out [Ly][Lx] FP64, indexed [n*Lx + m]; spec[0] = Lx*Ly.
 * Also makes this spectrum the context's current one. */
int cartogram_spectrum(cg_ctx* ctx, double* spec_out);

/* Density and velocity at diffusion time t from the current spectrum (SI Eq. rhoxyt
 * with Eq. fmn_diff, D = 1; v = -grad(rho)/rho): rho_out [Lx*Ly] (normalised density,
 * may be NULL), v_out [Lx*Ly][2] (vx, vy) at the cell centres. In mixed precision the
 * values are computed in FP32 and widened. */
int cartogram_velocity(cg_ctx* ctx, double t, double* rho_out, double* v_out);

/* One predictor-corrector step of all grid points from displacements disp_in
 * ([Lx*Ly][2], position = cell centre + displacement) with step h, using the fields
 * at times t and t+h of the current spectrum (main text: predictor-corrector with
 * bilinear interpolation). disp_out [Lx*Ly][2]; *err = max ||r_corr - r_pred||. */
int cartogram_heun_step(cg_ctx* ctx, double t, double h, const double* disp_in,
                        double* disp_out, double* err);

/* One integration (the step loop from t = 0 to equalisation) of the current spectrum.
 * grid_out [Lx*Ly][2] receives the projected cell centres (may be NULL); accepted and
 * rejected (may be NULL) the step counts, t_end the final time. Returns CG_OK or
 * CG_ESTEPFAIL. */
int cartogram_integrate_once(cg_ctx* ctx, double* grid_out, long long* accepted,
                             long long* rejected, double* t_end);

/* Diagnostic timing of the hot kernel classes on the context's stream with CUDA events:
 * each class is launched `reps` times on the current spectrum and the displacements
 * of the last integration, and ms_out[k] receives the mean device time per launch of
 *   0 inverse transform pass 1 (damping + rows), 1 inverse pass 2 (columns + velocity),
 *   2 predictor-corrector step of all grid points, 3 rasterisation (clear + edges + scan),
 *   4 forward transform (rows + columns), 5 vertex mapping + areas.
 * ms_out has 6 entries. Errors: CG_ESTATE (no map or no spectrum), CG_EINVAL. */
int cartogram_profile(cg_ctx* ctx, int reps, double* ms_out);

/* Pick the launch shapes of the three step kernels (spectral rows per block of the
 * first inverse pass, columns per block of the second, resident blocks per SM of the
 * predictor-corrector step) by timing each candidate `reps` times (best of three rounds)
 * with CUDA events on the context's stream, on the current spectrum and the
 * displacements of the last integration. reps = 0 changes nothing and only reports.
 * shapes_out[3] and ms_out[3] (may be NULL) receive the shapes in use and their mean
 * times per launch (0 if never timed). cartogram_integrate runs this once by itself,
 * after its first integration, when the autotune option is set. Errors: CG_EINVAL,
 * CG_ECUDA. */
int cartogram_autotune(cg_ctx* ctx, int reps, int* shapes_out, double* ms_out);

/* Diagnostic (no counterpart in the paper): the read bandwidth of the current GPU, the
 * roofline the step kernels are compared against. A buffer of `bytes` (from 1 MiB to
 * 64 GiB, a multiple of 16) is allocated, filled, read once, and then read `passes`
 * times by 8 blocks of 256 threads per SM with 16-byte loads that bypass L1, timed with
 * CUDA events (best of three). A buffer well below the L2 size measures L2 read
 * bandwidth, one far above it HBM read bandwidth. *gbs_out = bytes * passes / time in
 * GB/s (1e9 bytes). Synchronous. Errors: CG_EINVAL, CG_ENOMEM, CG_ECUDA. */
int cartogram_read_bandwidth(int64_t bytes, int passes, double* gbs_out);

/* Velocity field from a caller's spectrum with no device allocation. The paper has no
 * counterpart. It serves callers that cannot allocate GPU memory when they need the
 * field: a host application that gives this library a fixed device-memory budget and
 * owns every allocation itself, or a real-time loop that must not call the allocator
 * (cudaMalloc and cudaFree may synchronise the device and take unbounded time).
 *   Lx, Ly   powers of two from 8 to 512 (at most 512 x 512 cells); larger sizes
 *            return CG_EINVAL
 *   spec     device memory of the current device, FP32, [Ly][Lx] indexed [n*Lx + m],
 *            16-byte aligned: the cosine spectrum of rho/rho_bar - 1 (so spec[0] = 0),
 *            e.g. cartogram_spectrum's output with its (0,0) entry set to zero, rounded
 *            to FP32
 *   t        diffusion time (D = 1) at which the field is evaluated, >= 0
 *   v_out    device memory of the current device, FP32, [Lx*Ly][2] (vx, vy) at the cell
 *            centres, 16-byte aligned (the field is written with 16-byte stores)
 *   stream   cudaStream_t the work is queued on (NULL: the legacy default stream);
 *            the call returns without waiting for it
 * The scratch (about 2.1 MB: the intermediate of the two transform passes, the
 * transform tables and a reduction state) is one array in device memory created when
 * the library is loaded onto a GPU and kept until the process exits. The first call on
 * a device, with that device current, looks up the array's device address and sets
 * the kernels' shared-memory limits; make that first call before any stream capture
 * begins on the device. Every call on a device shares the array and
 * leaves its contents behind (the reduction state is cleared by each call): calls
 * whose work overlaps on the GPU (other streams, other host threads) race and must be
 * serialised by the caller. The call is asynchronous, so a failure inside the kernels
 * is not reported: a spectrum whose density is not positive everywhere gives a
 * meaningless field, as does a bounded wait inside the kernels that gave up. Returns
 * CG_OK, CG_EINVAL (sizes, NULL, alignment, host pointers or pointers of another
 * device) or CG_ECUDA; it calls no cudaMalloc, cudaFree or other allocating routine. */
int cartogram_velocity_noalloc(int Lx, int Ly, const float* spec, double t, float* v_out,
                               void* stream);

/* Description of the last error on this context ("" if none); valid until the next call. */
const char* cartogram_last_error(const cg_ctx* ctx);

/* Free the context and all its device memory. NULL is accepted. */
void cartogram_destroy(cg_ctx* ctx);

/* ---- Batches: many independent cartograms in one CUDA-graph launch --------------
 * The method's grid points are independent within one cartogram (main text: the
 * integrations of the Lx*Ly trajectories are distributed over processing units), and
 * separate cartograms (frames of an animation, replicates) are independent of each
 * other. A batch runs the outer iterations of several contexts as parallel branches
 * of one graph, so that the kernels of small grids share the GPU. */
typedef struct cg_batch cg_batch;

/* Group n contexts (distinct, on one device; sizes, precisions, flows and options may
 * differ). The batch refers to the contexts: destroy it before them. The batch graph
 * is captured on first use and again whenever a context's map or launch shapes
 * change. Errors: CG_EINVAL (n < 1, NULL or repeated context, devices differ),
 * CG_ECUDA. */
int cartogram_batch_create(cg_ctx* const* ctxs, int n, cg_batch** out);

/* cartogram_integrate for every context of the batch: contexts whose launch shapes are
 * still to be tuned first run one iteration on their own stream, then one launch of the
 * batch graph on the batch's stream runs all outer iterations (repeated while contexts
 * run out of history slots). stats[i] and status[i] (each [n] or NULL) receive every
 * context's outcome (seconds: the batch's wall time). Returns CG_OK when every context
 * converged, else the first failing context's status (message in
 * cartogram_batch_last_error; the context's own message in cartogram_last_error). */
int cartogram_batch_integrate(cg_batch* batch, cg_stats* stats, int* status);

/* Message of the last failed batch call. */
const char* cartogram_batch_last_error(const cg_batch* batch);

/* Free the batch (not its contexts). NULL is accepted. */
void cartogram_batch_destroy(cg_batch* batch);

#ifdef __cplusplus
}
#endif

#endif /* CARTOGRAM_H */
