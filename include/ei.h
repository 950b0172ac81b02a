/*
 * ei.h — C ABI of libei.so: model-based iterative reconstruction for x-ray
 * edge-illumination (EI) tomography on one NVIDIA GB300 (sm_103a), after
 * Modregger et al., "Accelerated iterative tomographic reconstruction with
 * x-ray edge illumination" (arXiv:2202.08627).
 *
 * The method ("Theoretical basis" section of the paper): for every slice, the
 * volumes mu (attenuation, 1/cm), delta (refractive decrement) and sigma
 * (scatter) are projected by the Radon transform R (Eq. 1); each detector
 * pixel's flat illumination curve (IC) f(t, m) is attenuated by exp(-R[mu]),
 * shifted by z d/dt R[delta] (Eq. 2; plus the drift m_o(theta) and ring term
 * m_r(t) of Eq. 4) and broadened by scatter, and evaluated at every mask
 * position m; the cost S of Eq. 5 (squared residual against the measured ICs
 * s_exp plus an L2 regulariser) is minimised with L-BFGS using its analytic
 * gradient.
 *
 * Discretisation (the paper leaves it open; this library's reading):
 *   - voxel (r, c) of an n x n slice is centred at x = (c - (n-1)/2) pitch,
 *     y = ((n-1)/2 - r) pitch; detector pixel j at t_j = (j - (n_det-1)/2) pitch;
 *     angle theta_a = a pi / n_theta unless given; ray {x cos + y sin = t}.
 *   - R: ray-driven linear interpolation ("Algorithmic improvements"
 *     section: linear interpolation, indices computed on the fly), one sample
 *     per voxel row (column when |sin| > |cos|), weight pitch / max(|cos|,|sin|).
 *   - d/dt: central finite differences, one-sided at the detector ends
 *     ("Experimental improvements" section).
 *   - IC: f(t, m) = A_t exp(-(m - c_t)^2 / (2 w_t^2)) (Gaussian flat IC per
 *     pixel, m in mask periods); with V = w_t^2 + kappa R[sigma] and
 *     shift = (z / period) dR[delta]/dt + m_o(theta) + m_r(t):
 *       s_mod = exp(-R[mu]) A_t (w_t / sqrt(V)) exp(-(m - c_t - shift)^2 / (2 V)).
 *   - S = sum (s_exp - s_mod)^2 + sum_c lambda_c ||x_c / scale_c||^2, and
 *     S = +inf where V <= 0.01 w_t^2 (outside the model's domain).
 *
 * Memory layout (all float32 unless stated; slices are stored one after the
 * other in slice order, the offsets are reported by ei_get_slice_layout):
 *   vol    per slice n*n float4 = (mu, delta, sigma, pad), row-major [r][c].
 *          The pad lane is ignored on input and written as 0 on output.
 *   proj   per slice 3 planes [channel][n_theta][n_dp], channel = mu, delta, sigma.
 *   sino4  per slice [n_theta][n_dp] float4 = (mu, delta, sigma, pad).
 *   s_exp, s_mod  per slice n_m planes [m][n_theta][n_dp].
 *   n_dp = n_det rounded up to a multiple of 4; pixels n_det..n_dp-1 are
 *   padding: ignored on input, written as 0 on output.
 *   Every array pointer must be 16-byte aligned.
 *
 * Ownership: every array argument is caller-owned.  Unless a function says
 * otherwise, array pointers are DEVICE pointers (cudaMalloc'd or a PyTorch
 * CUDA tensor's storage) on the current device.  The geometry handle owns its
 * own device workspace (allocated in ei_setup_geometry and ei_reconstruct,
 * freed in ei_destroy_geometry).
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls are stream-ordered and asynchronous unless stated.  A
 * geometry's workspace is shared by its calls, so calls on one geometry must
 * not overlap on the GPU (use one stream per geometry, or synchronise).
 *
 * Errors: every function returns an ei_status; nothing is thrown across the
 * ABI.  EI_ERR_ARG is returned before any work is queued.  After EI_ERR_CUDA
 * the contents of output arrays are unspecified.
 */
#ifndef EI_H
#define EI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EI_OK = 0,
    EI_ERR_ARG = 1,          /* invalid argument (null, size, layout, alignment) */
    EI_ERR_CUDA = 2,         /* a CUDA call failed (launch, copy, allocation) */
    EI_ERR_NONFINITE = 3,    /* the objective is NaN (non-finite data or iterate) */
    EI_ERR_LINESEARCH = 4,   /* Armijo backtracking found no acceptable step */
    EI_ERR_TIMEOUT = 5,      /* a kernel's bounded wait ran out, or a solve's time budget
                                (ei_solve_opts.max_seconds) did */
    EI_ERR_DEVICE_CHECK = 6, /* a kernel's index bounds check fired (only the build with
                                device checks, libei_check.so, has them) */
    EI_ERR_ALLOC = 7         /* workspace allocation failed */
} ei_status;

typedef struct ei_geometry ei_geometry;   /* opaque */

/* Per-slice sizes for batches of uneven slices. */
typedef struct {
    int n;            /* slice is n x n voxels, n >= 1 */
    int n_theta;      /* projection angles, >= 1 */
    int n_det;        /* detector pixels, 1 <= n_det <= EI_MAX_NDET */
    double pitch_cm;  /* voxel pitch = detector pitch (cm), > 0 */
} ei_slice_dims;

#define EI_MAX_NDET 8192
#define EI_MAX_NM 32

/*
 * Acquisition geometry and model constants (Eq. 2, Eq. 4, Eq. 5).
 * Host arrays are copied during ei_setup_geometry; flat_* / m_o / m_r may be
 * host or device pointers (copied too).
 */
typedef struct {
    int n, n_theta, n_det;     /* uniform batch: every slice n x n, n_theta angles, n_det pixels */
    int n_m;                   /* mask positions M, 1 <= M <= EI_MAX_NM (all slices) */
    double pitch_cm;           /* uniform batch: voxel = detector pitch (cm) */
    const double *theta;       /* host; NULL = theta_a = a pi / n_theta.  Uniform batch:
                                  [n_theta]; uneven batch: concatenated per slice */
    const double *m;           /* host [n_m]: mask positions in IC periods */
    double z_cm;               /* sample-detector distance z (cm) */
    double period_cm;          /* IC period the shift is expressed in: shift = (z/period) dR[delta]/dt */
    double kappa_sigma;        /* IC variance (period^2) added per unit of R[sigma] */
    const float *flat_A;       /* Gaussian flat IC per pixel: amplitude, centre (periods), */
    const float *flat_c;       /* width w > 0 (std, periods).  Uniform batch: [n_det] shared */
    const float *flat_w;       /* by all slices; uneven batch: concatenated [n_det_s] per slice */
    double lambda[3];          /* L2 weights (mu, delta, sigma); the paper uses 1e-2 */
    double scale[3];           /* variable scaling u = x / scale for the solver and the
                                  regulariser (e.g. 1, 1e-6, 1); > 0 */
    const float *m_o;          /* optional drift m_o(theta) per angle (Eq. 4), NULL = 0;
                                  layout like theta */
    const float *m_r;          /* optional ring term m_r(t) per pixel (Eq. 4), NULL = 0;
                                  layout like flat_* */
} ei_geometry_desc;

/*
 * Build a geometry for a batch of n_slices slices and allocate its workspace
 * on the current device.  per_slice == NULL: every slice takes desc->n,
 * n_theta, n_det, pitch_cm.  Otherwise per_slice[n_slices] gives each slice's
 * sizes (desc->n .. pitch_cm are ignored) and the per-slice arrays described
 * above are concatenated in slice order.
 * Returns EI_ERR_ARG on invalid sizes or constants, EI_ERR_ALLOC/EI_ERR_CUDA
 * when the workspace cannot be allocated.  Synchronous.
 */
int ei_setup_geometry(const ei_geometry_desc *desc, int n_slices,
                      const ei_slice_dims *per_slice, ei_geometry **out);

/* Free a geometry and its workspace (synchronises the device first).  NULL is a no-op. */
void ei_destroy_geometry(ei_geometry *g);

/* Sizes of one slice's arrays, in ELEMENTS of the array's element type, and
 * the element offset of the slice inside each batched array. */
typedef struct {
    int n, n_theta, n_det, n_dp, n_m;
    double pitch_cm;
    int64_t vol_offset, vol_count;     /* float4 elements */
    int64_t proj_offset, proj_count;   /* floats (3 planes) */
    int64_t sino4_offset, sino4_count; /* float4 elements */
    int64_t meas_offset, meas_count;   /* floats (n_m planes): s_exp, s_mod */
} ei_slice_layout;

/* Totals for the whole batch, same units. */
typedef struct {
    int n_slices, n_m;
    int64_t vol_count, proj_count, sino4_count, meas_count;
    int64_t workspace_bytes;           /* device bytes the geometry holds */
} ei_layout;

int ei_get_layout(const ei_geometry *g, ei_layout *out);
int ei_get_slice_layout(const ei_geometry *g, int slice, ei_slice_layout *out);

/*
 * proj = R[vol] for the three channels of every slice (Eq. 1).
 * vol: device, vol layout; proj: device, proj layout.
 */
int ei_project(const ei_geometry *g, const float *vol, float *proj, void *stream);

/*
 * vol = R^T[sino4] for the three channels of every slice: the transpose of
 * ei_project, which the analytic gradient of Eq. 5 needs.  Gather form, no
 * atomics.  sino4: device, sino4 layout; vol: device, vol layout.
 */
int ei_backproject(const ei_geometry *g, const float *sino4, float *vol, void *stream);

/*
 * s_mod = IC model (Eq. 2 with the Eq. 4 offsets and scatter broadening)
 * evaluated from given projections.  proj: device, proj layout;
 * s_mod: device, measurement layout.
 */
int ei_ic_model(const ei_geometry *g, const float *proj, float *s_mod, void *stream);

/*
 * Non-iterative (single-shot) reconstruction, the warm-start input of the
 * iteration: the paper's non-iterative baseline retrieves the projection from
 * a single mask position (Eq. 3) and inverts it with a filtered
 * back-projection.  Here, per pixel, the moments over m of s_exp against the
 * flat IC give R[mu] = -ln(sum s / sum f), the IC shift (centroid difference,
 * minus m_o and m_r), integrated along t into R[delta] with both row ends
 * pinned to zero, and R[sigma] = max(0, var s - var f) / kappa; each channel
 * is Ram-Lak filtered along t and back-projected (pi / n_theta / pitch R^T).
 * s_exp: device, measurement layout; vol_out: device, vol layout (physical).
 */
int ei_single_shot_fbp(const ei_geometry *g, const float *s_exp, float *vol_out, void *stream);

/* s_mod for a physical volume: ei_project followed by ei_ic_model. */
int ei_forward(const ei_geometry *g, const float *vol, float *s_mod, void *stream);

/*
 * S (Eq. 5) of every slice and, if grad != NULL, its gradient with respect to
 * the physical volume:
 *   S_s    = sum_{t,theta,m} (s_exp - s_mod)^2 + sum_c lambda_c ||x_c / scale_c||^2
 *   grad_c = R^T[dS/dR[x_c]] + 2 lambda_c x_c / scale_c^2
 * vol, s_exp, grad: device (vol / measurement / vol layout).
 * S_out: [n_slices] doubles, host or device memory.  The data term is
 * accumulated in FP64 in a fixed order (deterministic).  When S_out is host
 * memory the call synchronises the stream before returning.
 * A slice outside the model's domain reports S = +inf; a NaN in s_exp or vol
 * reports NaN (the call itself still returns EI_OK).
 */
int ei_objective_grad(const ei_geometry *g, const float *vol, const float *s_exp,
                      double *S_out, float *grad, void *stream);

/* L-BFGS options ("Theoretical basis" section: L-BFGS as in SciPy [Byrd 1995]). */
typedef struct {
    double tol;        /* stop when (f_k - f_k+1) / max(|f_k|, |f_k+1|, 1) < tol (e.g. 1e-6) */
    int max_iter;      /* accepted steps per slice */
    int lbfgs_m;       /* (s, y) pairs kept, 1..32 (SciPy default 10) */
    double c1;         /* Armijo constant (1e-4) */
    int max_trials;    /* step halvings per line search (20) */
    double curv_eps;   /* keep a pair only if s.y > curv_eps |s| |y| (1e-10) */
    int use_graph;     /* 1: capture one solver round into a CUDA graph and replay it (1) */
    int resume;        /* 1: continue from the solver state instead of starting at vol_inout (0);
                          see ei_solver_save / ei_solver_load */
    double max_seconds; /* wall-clock budget of the call, 0 = none (0).  Checked on the host
                          before each solver round, when no work of the call is in flight:
                          once it has run out the call stops, the slices still iterating
                          report EI_ERR_TIMEOUT and return their last accepted iterate, and
                          the kept solver state is left as it was, so a call with resume = 1
                          continues them exactly where they stopped */
} ei_solve_opts;

/* Per-slice results; every pointer is a caller-owned HOST array of n_slices
 * entries, or NULL when not wanted. */
typedef struct {
    int *iterations;   /* accepted steps */
    int *status;       /* ei_status per slice: EI_OK (converged or max_iter reached),
                          EI_ERR_LINESEARCH, EI_ERR_NONFINITE, EI_ERR_TIMEOUT (still
                          iterating when max_seconds ran out) */
    int *converged;    /* 1 if the tol test stopped the slice, 0 if max_iter or an error did */
    double *f_final;   /* final S */
    double *f_initial; /* S at x0 */
    int *slice_evaluations; /* objective evaluations of each slice (every line-search
                          trial and the initial point) */
    int evaluations;   /* batched evaluation rounds, the initial one included (out) */
    double seconds;    /* wall time of the call (out) */
    int *slice_projections; /* forward projections of each slice: the initial point and
                          the first trial of every iteration (a backtracking trial's
                          projections are interpolated, R being linear) */
    int *slice_adjoints; /* adjoint back-projections of each slice: the initial point and
                          every accepted step */
} ei_solve_report;

/*
 * Minimise S (Eq. 5) for every slice independently with batched L-BFGS:
 * two-loop recursion with H0 = (s.y / y.y) I, Armijo backtracking (first
 * trial 1/|g| while no pair is kept, then 1, halving), pair kept when the
 * curvature condition holds, stop on the relative decrease of S or max_iter.
 * The iterate is u = x / scale.  R is linear, so along a search direction
 * the projections of u + alpha d are P(u) + alpha P(d): each iteration
 * projects its first trial point only, a backtracking trial interpolates
 * between the projections of u and of the previous trial (a rejected trial
 * costs the IC model alone), and the adjoint runs at accepted points only
 * (the "Algorithmic improvements" section's removal of superfluous Radon
 * calls).
 * s_exp: measurement layout, vol_inout: vol layout (x0 in, solution out);
 * both may be device or host memory (host arrays are staged through device
 * memory inside the call).  report may be NULL.  Synchronous: `stream` is
 * synchronised first, the iterations run on a stream the solver owns (one
 * solver round is captured into a CUDA graph and replayed), and the call
 * returns when every slice has stopped or max_seconds has run out.  Returns EI_OK
 * when every slice converged or reached max_iter, else the first per-slice error;
 * EI_ERR_ARG for invalid options (max_seconds negative or NaN among them).
 */
int ei_reconstruct(const ei_geometry *g, const float *s_exp, float *vol_inout,
                   const ei_solve_opts *opts, ei_solve_report *report, void *stream);

/* Default options: tol 1e-6, max_iter 100, m 10, c1 1e-4, 20 trials, 1e-10, graphs on,
 * no resume, no time budget. */
void ei_default_solve_opts(ei_solve_opts *opts);

/*
 * Checkpoint / resume of the solver.  After ei_reconstruct returns, the
 * geometry keeps the L-BFGS state of every slice: the iterate u = x / scale
 * and its gradient, the search direction, the m most recent (s, y) pairs and
 * their 1 / s.y, the projections of u and of the latest trial point, the
 * accepted-step count k, the current and initial S, and whether the slice
 * converged, failed, or is between steps.
 *   ei_solver_state_size: bytes of that state for this geometry and lbfgs_m.
 *   ei_solver_save: copies it to buf (host or device, >= the size); EI_ERR_ARG
 *     when no ei_reconstruct call has returned its state on this geometry (a
 *     call stopped by its time budget does).
 *   ei_solver_load: installs a saved state in a geometry of the same slices,
 *     unknowns (linked mode, offsets) and lbfgs_m; EI_ERR_ARG when the header
 *     does not match.
 * ei_reconstruct with opts.resume = 1 then continues from the state (vol_inout
 * is output only, s_exp must be the same data): slices that stopped at
 * max_iter resume with the new max_iter (k counts from the original start),
 * converged or failed slices stay so, and the iterates are bit-identical to
 * one uninterrupted solve with the larger max_iter.  The state holds
 * (2 m + 5) vectors of the volume's size, two sets of the three projection
 * planes, and small per-slice records.
 */
int ei_solver_state_size(const ei_geometry *g, int lbfgs_m, size_t *bytes);
int ei_solver_save(const ei_geometry *g, void *buf, size_t bytes);
int ei_solver_load(ei_geometry *g, int lbfgs_m, const void *buf, size_t bytes);

/*
 * Tracing: per-kernel CUDA-event timings and a count of every kernel this
 * library launches.  ei_profile_enable(g, 1) resets the counters and starts
 * recording events around the projector, IC and adjoint launches (on the
 * stream they run on); 0 resets the counters and stops recording events (the
 * launch count goes on).  While events are recorded, ei_reconstruct runs its
 * rounds without CUDA-graph replay so that every launch is timed.  ei_profile_read synchronises the
 * device and sums the recorded durations.  Not part of the paper's method.
 */
typedef struct {
    int64_t launches;              /* all kernels launched while enabled */
    int64_t project_launches, ic_launches, backproject_launches;
    double project_ms, ic_ms, backproject_ms;   /* summed event durations */
} ei_profile;

int ei_profile_enable(ei_geometry *g, int on);
int ei_profile_read(ei_geometry *g, ei_profile *out);

/*
 * Kernel variants and autotuning (batched, serving-style launches).
 * The projector and the adjoint each come in several tile shapes
 * (projector, rays x angles per block / per warp and samples per loop
 * iteration, lanes ray-major: 0 16x16/8x4/4, 1 32x8/8x4/4, 2 32x16/8x4/4,
 * 3 16x16/8x4/2, 4 32x8/32x1/4, 5 16x16/16x2/4, 6 32x16/32x1/4; lanes
 * angle-major: 7 16x16/4x8/4, 8 8x32/4x8/4, 9 32x8/4x8/4, 10 16x16/2x16/4;
 * lanes in groups of 8 on 2 rays x 4 angles: 11 8x32/4x8/4, and 12 the same
 * with groups of 16 on 4 rays x 4 angles; 13 32x32 with each thread on 4 rays
 * of one angle and warps on 4 rays x 8 angles, whose rows are staged in shared
 * memory by bulk asynchronous copies (one block per work item in every launch
 * mode; blocks mixing row- and column-first angles load from global memory);
 * adjoint: 0 8, 1 4, 2 16 voxels per
 * thread with lanes along rows of 8 voxels, 3 8 and 4 16 voxels per thread
 * with 8-lane groups on 2 x 4 sub-patches, 5-7 four pairs of horizontally
 * adjacent voxels per thread (the pair shares its three detector pixels per
 * angle) with lanes along rows of 16 voxels, on 4 x 4 sub-patches in warps of
 * 16 x 4, or in warps of 8 x 8, 8-10 a pair of the slice's top-left quadrant
 * and its three mirror images about the slice centre (a point mirror takes
 * the same hat weights at the mirrored pixels), in 16 or 32 rows per tile,
 * 11-13 the same over gradient rows whose entry j holds pixel j and its
 * mirror pixel n_det - 1 - j, a voxel and its point mirror advanced by one
 * paired FP32 FMA (fma.rn.f32x2; results equal those of 8-10 bit for bit)),
 * launched in one of three modes (the `persistent` argument): 0 one block
 * per work item, 1 a persistent GPU-sized grid whose blocks take work items
 * from one counter, 2 a persistent grid whose blocks first take the items of
 * their own SM's contiguous chunk of the work list (the blocks resident on an
 * SM then work on neighbouring items and share L1 lines), then those of the
 * other chunks.  Projector variants compute every
 * ray identically (bit-identical projections); adjoint variants sum every
 * voxel's angles in the same order but round the detector coordinate from a
 * different tile origin, so gradients agree to FP32 rounding (~1e-7
 * relative).  Launch mode and graph replay never change results.
 *
 * ei_autotune times every candidate with CUDA events on this geometry's
 * workspace (synchronises `stream`) and selects the fastest; the choice is
 * cached in a text file (EI_TUNE_CACHE, default ~/.cache/ei_gb300_autotune.txt)
 * keyed by the GPU name, the slice sizes, whether the geometry is linked
 * (ei_set_linked: the single-channel kernels are timed) and the number of
 * variants this build has, and read back on later calls
 * unless EI_TUNE_FORCE is set.  ei_set_variant / ei_get_variant select and
 * report a variant explicitly (ids: projector 0..13, adjoint 0..13, launch
 * mode 0..2).
 */
#define EI_TUNE_FORCE 1
#define EI_TUNE_NO_CACHE_WRITE 2
int ei_autotune(ei_geometry *g, int flags, void *stream);
int ei_set_variant(ei_geometry *g, int fwd_variant, int adj_variant, int persistent);
int ei_get_variant(const ei_geometry *g, int *fwd_variant, int *adj_variant, int *persistent);

/*
 * Linked single unknown of Eq. 4.  With gamma > 0 the geometry models
 * mu = h, delta = gamma h, sigma = 0 (the paper's homogeneous-sample
 * assumption): ei_forward, ei_objective_grad, ei_offset_grad and
 * ei_reconstruct read h from the mu lane of the volume (the other lanes are
 * ignored), gradients come back as (dS/dh, 0, 0, 0), ei_reconstruct returns
 * (h, 0, 0, 0), and the regulariser is lambda[0] ||h / scale[0]||^2 (the
 * paper's lambda ||h||^2).  gamma is delta / mu in cm (the paper's gamma = 5 is
 * in units it does not state).  gamma = 0 restores three independent channels.
 * ei_project and ei_backproject stay the plain linear operators.  EI_ERR_ARG
 * for a negative or non-finite gamma.
 */
int ei_set_linked(ei_geometry *g, double gamma);

/*
 * The paper's single-shot retrieval (Eq. 3), for the homogeneous-sample model
 * mu = h, delta = gamma h (gamma in cm, as for ei_set_linked), from the one
 * mask position m_index of s_exp (an acquisition on the slope of the IC; other
 * positions are not read), then the filtered back-projection.  Reading of
 * Eq. 3: linearising Eq. 4 at m gives s / f = (1 + a d/dt) T with
 * T = exp(-R[h]) and a = (z/period) gamma f'(m) / f(m), f the flat IC averaged
 * over the slice's pixels; Eq. 3 divides by (1 + i q a) in Fourier space along
 * t, computed here as the equivalent circular convolution with the real DFT
 * kernel.  R[h] = -ln T (T clamped at 1e-6), ramp filter, FBP.
 * vol_out: (h, gamma h, 0, 0) per voxel.  Offsets m_o, m_r are not modelled.
 * EI_ERR_ARG for m_index outside [0, n_m), a negative or non-finite gamma, or
 * rows wider than 6257 pixels.  The first call allocates one float per
 * detector pixel.
 */
int ei_single_shot_eq3(ei_geometry *g, const float *s_exp, int m_index, double gamma,
                       float *vol_out, void *stream);

/*
 * Gradient of S (Eq. 5) with respect to the drift m_o(theta) and the ring
 * term m_r(t) of Eq. 4, at the physical volume vol (layout of ei_forward).
 * Both terms enter only the shift of pixel (theta, t), with coefficient 1:
 *   dS/dm_o(theta) = sum_t dS/dshift,   dS/dm_r(t) = sum_theta dS/dshift,
 *   dS/dshift = sum_m 2 (s_mod - s_exp) s_mod q / V    (q = m - c - shift),
 * each sum accumulated in FP64 in a fixed order.  g_mo: device [sum n_theta],
 * g_mr: device [sum n_det], per slice in slice order (for a uniform batch whose
 * m_o / m_r are shared by every slice, the gradient of the shared array is the
 * sum over slices); either may be NULL.  Values are unspecified where S is
 * +inf.  The first call allocates one float per sinogram pixel of scratch;
 * stream-ordered otherwise.  With a sampled flat IC (ei_set_flat_table)
 * dS/dshift = sum_m 2 (s_mod - s_exp) (-exp(-R[mu]) f'(m - shift)).
 * ei_set_offset_unknowns makes m_o / m_r unknowns of ei_reconstruct.
 */
int ei_offset_grad(ei_geometry *g, const float *vol, const float *s_exp, float *g_mo, float *g_mr,
                   void *stream);

/*
 * Eq. 4's offsets as unknowns of ei_reconstruct (the paper minimises S over
 * h, m_o and m_r together).  which = EI_OFFSET_MO | EI_OFFSET_MR selects the
 * drift m_o(theta) and / or the ring term m_r(t) of every slice; the solver
 * iterates on m / scale (scale > 0, in IC periods) starting from the
 * geometry's current values (ei_setup_geometry's m_o / m_r, per slice), and
 * leaves the solution's offsets in the geometry, where every later call uses
 * them and ei_get_offsets reads them.  When both are unknowns, the gauge
 * (m_o + a, m_r - a), which leaves S unchanged, is fixed by keeping the mean
 * of m_r over each slice's pixels at its starting value (its gradient is
 * projected onto zero mean).  which = 0 restores fixed offsets.  Each solver
 * evaluation then also computes dS/dshift per pixel (one more pass over the
 * projections and measured ICs).
 */
#define EI_OFFSET_MO 1
#define EI_OFFSET_MR 2
int ei_set_offset_unknowns(ei_geometry *g, int which, double scale);

/*
 * Restrict the ring term m_r(t) of Eq. 4, when it is among the solver's
 * unknowns, to pixel-to-pixel (ring) frequencies: each slice's m_r gradient
 * is projected onto the orthogonal complement of the K lowest orthonormal
 * DCT-II modes across its detector,
 *   b_k(j) = sqrt((2 - [k = 0]) / n_det) cos(pi k (j + 1/2) / n_det),  k < K,
 * so m_r keeps its starting component in those modes.  A ring artefact is a
 * per-pixel error of the flat IC, present at every frequency, while the shift
 * that the object's angle-averaged projection causes varies slowly across
 * the detector: a free m_r absorbs that part of the object's signal too (the
 * paper's "Experimental improvements" section introduces m_r against rings;
 * the restriction is this library's reading).  K = 0 (the default): no
 * restriction beyond the zero-mean gauge of ei_set_offset_unknowns; K >= 1
 * includes that gauge.  0 <= K <= EI_MAX_RING_MODES and K <= every slice's
 * n_det, else EI_ERR_ARG.  Takes effect from the next ei_reconstruct call.
 */
#define EI_MAX_RING_MODES 1024
int ei_set_ring_modes(ei_geometry *g, int K);
/* The geometry's current m_o [sum n_theta] and m_r [sum n_det], per slice in
 * slice order, into host or device arrays (either may be NULL).  Synchronous. */
int ei_get_offsets(const ei_geometry *g, float *m_o, float *m_r);

/*
 * Sampled flat IC.  The paper's flat IC is measured by stepping the mask over
 * one period (acquisition section); instead of its Gaussian fit (flat_A,
 * flat_c, flat_w of ei_setup_geometry) the model can use the samples
 * themselves:  s(t, theta, m) = exp(-R[mu]) f_t(m - shift),  shift as in
 * Eq. 4, with f_t interpolated in m by periodic cubic Catmull-Rom splines
 * through table[t][k] = f_t(k / K), k = 0 .. K-1 (m in periods, period 1).
 * table: host or device pointer, [sum n_det][K] floats row-major, pixels in
 * the order of flat_A (slice by slice); copied into the geometry, which
 * keeps no reference, after a device synchronisation (no kernel may be
 * reading the previous table).  R[sigma] has no effect in this model:
 * its gradient is 0 and V's domain check is off.  Affects ei_ic_model,
 * ei_forward, ei_objective / ei_objective_grad, ei_offset_grad and
 * ei_reconstruct (which run the one-block-per-row IC kernel while a table is
 * set); the single-shot retrievals keep the Gaussian parameters.  table =
 * NULL or K = 0 restores the Gaussian.  EI_ERR_ARG for K outside
 * [4, 65536]; EI_ERR_ALLOC / EI_ERR_CUDA when the copy fails, after which
 * the Gaussian flat is in effect.
 */
int ei_set_flat_table(ei_geometry *g, const float *table, int K);

/*
 * On-chip throughput of the current GPU, measured by microbenchmarks (each the
 * best of three CUDA-event-timed runs after a warm-up; ~10 ms in all): the
 * FP32 FMA rate (2 flops per FMA), the rate at which 16-byte global loads that
 * hit L1 deliver bytes to registers, and the same for shared-memory loads.
 * They are the denominators of the rooflines of kernels bound on chip rather
 * than by HBM.  The paper has no counterpart.  Synchronises `stream`;
 * allocates and frees 8 KB of device memory.
 */
typedef struct {
    double fp32_tflops;
    double l1_load_tbs;      /* TB/s, all SMs */
    double smem_load_tbs;    /* TB/s, all SMs */
    int num_sms;
} ei_peaks;
int ei_measure_peaks(ei_peaks *out, void *stream);

/*
 * Failure-detection self-test of the bounded waits.  The bulk-copy kernels
 * (the IC pipeline, the tensor-core convolutions) wait on mbarriers for at
 * most a fixed time and then report EI_ERR_TIMEOUT through a device status
 * word instead of hanging.  This runs that wait on an mbarrier that nothing
 * ever completes, limited to limit_us microseconds (1 .. 2e6), on the current
 * device (synchronous), and stores the status the kernel recorded in
 * *status_out: EI_ERR_TIMEOUT when the wait gave up as it must.  Returns
 * EI_ERR_ARG for a bad limit or NULL status_out, EI_ERR_CUDA if the launch or
 * copy failed; the CUDA context stays usable.
 */
int ei_selftest_wait_timeout(unsigned limit_us, int *status_out);

/*
 * Debug build with device-side bounds checks (SURVEY-style sanitizer
 * stand-in; the library built with -DEI_DEVICE_CHECKS as libei_check.so).
 * The projector and the adjoint index the packed volume and gradient rows
 * through zero margins sized on the host, without checks; in the check build
 * every such data-dependent index is verified, a failed check stores
 * EI_ERR_DEVICE_CHECK in the geometry's device status word (returned by the
 * next synchronising call: ei_reconstruct, or ei_objective_grad with a host
 * S_out) and the access is clamped into its array.  Results are otherwise
 * bit-identical to the regular build's.
 *   ei_device_checks_enabled: 1 in the check build, 0 otherwise.
 *   ei_selftest_device_check: runs a checked read whose index leaves its
 *     logical range but not its buffer (synchronous, on the current device)
 *     and stores the recorded status in *status_out: EI_ERR_DEVICE_CHECK in
 *     the check build, 0 in the regular one.  EI_ERR_ARG for NULL, EI_ERR_CUDA
 *     if the launch or copy failed.
 */
int ei_device_checks_enabled(void);
int ei_selftest_device_check(int *status_out);

/*
 * Failure injection on the host, for testing the clean-up paths.  Every
 * device allocation the library makes for a geometry, its solver and a U-Net
 * goes through one allocator that counts the live allocations.
 *   ei_fail_alloc_after(n), n >= 0: the next n allocations succeed and the
 *     one after them fails as if the device were out of memory (the call that
 *     made it then returns EI_ERR_ALLOC after freeing what it had allocated);
 *     the trigger is then disarmed.  n = -1 disarms it.  Process-wide.
 *     EI_ERR_ARG for n < -1.
 *   ei_fail_alloc_pending(*n): the allocations still to pass before the
 *     armed failure, or -1 when none is armed (it fired or was disarmed).
 *   ei_live_allocations(*n): device allocations currently held by the
 *     library (all geometries and networks).  EI_ERR_ARG for NULL.
 * No kernel, device fault or GPU state is involved.
 */
int ei_fail_alloc_after(int n);
int ei_fail_alloc_pending(int *n);
int ei_live_allocations(int64_t *n);

/*
 * IC kernel variant (the fused Eq. 2 model, Eq. 5 residual and gradient).
 *   0: one block per sinogram row; any row width and M.
 *   1: persistent blocks (as many as fit on the GPU) that stream rows through
 *      NST shared-memory buffers filled by bulk asynchronous copies, so the
 *      reads of the next NST - 1 rows overlap the arithmetic of the current
 *      one.  NST = 3 when (3 (3 + M) + 3) * 4 * max n_dp bytes <= 220 KB (rows
 *      up to 1536 pixels with M = 7), else 2 when (2 (3 + M) + 3) * 4 * max n_dp
 *      bytes fit; EI_ERR_ARG otherwise.
 * ei_setup_geometry selects 1 when it fits, else 0.  The two agree to FP32
 * rounding (variant 1 evaluates the exponential as 2^(log2(e) x) with the
 * PTX ex2 instruction).  Variant 1's waits for its copies are bounded (2 s);
 * a wait that runs out poisons the affected slices' objectives with NaN and
 * sets a device status word, which the synchronous calls (ei_objective_grad
 * with a host S_out, ei_reconstruct) return as EI_ERR_TIMEOUT.
 */
int ei_set_ic_variant(ei_geometry *g, int variant);
int ei_get_ic_variant(const ei_geometry *g, int *variant);

/*
 * Learned warm start (not in the paper): a U-Net that maps
 * the single-shot reconstruction (ei_single_shot_fbp, in the solver's scaled
 * units u = x / scale) to a start near the converged iteration, y = x + net(x).
 * levels L (1..6), base width 32 or 64 (width of level l: base 2^l); per
 * encoder level two 3x3 conv + ReLU (2x2 average pooling between levels), per
 * decoder level a nearest 2x upsample, 3x3 conv + ReLU, 3x3 conv + ReLU over
 * the concatenation with the skip tensor, 3x3 conv + ReLU; a 1x1 head.  BF16
 * activations and tensor-core convolutions with FP32 accumulation (tcgen05
 * with the accumulator in tensor memory, or WMMA mma.sync: see
 * ei_unet_set_tensor_path), FP32 master weights updated by Adam
 * (0.9, 0.999, 1e-8).  height and width must
 * be multiples of 2^(L-1); every batch is at most the `batch` of creation.
 * Arrays: x, y, target are device FP32 NHWC [batch][height][width][3].
 * Parameters (export order): each conv's W [tap][c_in][c_out] then b [c_out]
 * in creation order (encoder levels 0..L-1: two convs each; decoder levels
 * L-2..0: up-conv, concat-conv, conv), then head W [base][3], head b [3].
 */
typedef struct ei_unet ei_unet;
int ei_unet_create(int levels, int base, int batch, int height, int width,
                   unsigned long long seed, ei_unet **out);
void ei_unet_destroy(ei_unet *net);
int ei_unet_forward(ei_unet *net, const float *x, float *y, int batch, void *stream);
/* one Adam step on the MSE loss mean((y - target)^2); *loss (host, may be NULL)
 * receives the loss before the step (synchronises the stream when non-NULL) */
int ei_unet_train_step(ei_unet *net, const float *x, const float *target, int batch, double lr,
                       double *loss, void *stream);
int64_t ei_unet_num_params(const ei_unet *net);
/* host arrays of ei_unet_num_params floats (synchronous) */
int ei_unet_get_params(const ei_unet *net, float *host);
int ei_unet_set_params(ei_unet *net, const float *host);
int ei_unet_get_grads(const ei_unet *net, float *host);
/* Adam's state for a training checkpoint: the first and second moments
 * (host arrays of ei_unet_num_params floats, the parameters' order) and the
 * step count; with the parameters (ei_unet_get_params / _set_params) a restored
 * network continues training bit-identically.  Synchronous. */
int ei_unet_get_optimizer(const ei_unet *net, float *m_host, float *v_host, int *step);
int ei_unet_set_optimizer(ei_unet *net, const float *m_host, const float *v_host, int step);
/* Convolution path: 1 (default) tcgen05 implicit-GEMM kernels for the forward
 * pass, the input gradients and the weight gradients of every convolution whose
 * channel counts they support (input channels a multiple of 32; output channels
 * 32, 64, 128 or a multiple of 256); 0 the WMMA (mma.sync) kernels for all.  Both accumulate in FP32; results agree to FP32 rounding of
 * the sums.  A tcgen05 kernel whose bounded wait runs out makes the next
 * synchronising ei_unet_train_step return EI_ERR_TIMEOUT. */
int ei_unet_set_tensor_path(ei_unet *net, int path);

/*
 * ei_objective_grad_noalloc — S and its gradient for ONE slice with no device
 * allocation at all.  The paper has no counterpart; this exists for callers
 * that may not allocate GPU memory themselves: frameworks that have reserved
 * the device memory for their own pool and forbid allocations outside it, and
 * latency-sensitive loops that cannot afford cudaMalloc's implicit device
 * synchronisation.  Such callers cannot use ei_setup_geometry (it allocates a
 * workspace), so the geometry description is passed directly.
 *
 * desc: as for ei_setup_geometry with a uniform batch of one slice (desc->n,
 *   n_theta, n_det, pitch_cm; flat_*, m_o, m_r host or device), checked as
 *   ei_setup_geometry checks it (flat_w > 0, finite flat_A and flat_c, finite
 *   constants), device arrays included: they are read back through `stream`.
 * vol, s_exp, grad (nullable), S_out: as for ei_objective_grad, one slice.
 * Kernels: variant 0 of the projector, the IC kernel and the adjoint, so the
 *   results equal those of ei_objective_grad on a geometry of the same slice
 *   set to those variants (ei_set_variant(g, 0, 0, 0), ei_set_ic_variant(g, 0)).
 * Scratch: every intermediate lives in one static device array of
 *   EI_NOALLOC_SCRATCH_BYTES that each GPU loading the library holds until the
 *   process exits.  A slice needs about 48 n(n+1) + 12 n_theta n_dp
 *   + 24 n_theta (n_dp + 2 margin) bytes plus small tables (margin ~
 *   max(2, 0.71 n - n_det/2 + 3) pixels); larger slices return EI_ERR_ARG
 *   before any GPU work.  (A 256x256 slice with 720 angles and 384 pixels
 *   needs ~14 MB.)
 * Every call looks up the array's address in the current context
 *   (cudaGetSymbolAddress) and sets the IC kernel's shared-memory limit; no
 *   state is kept between calls but the array's contents.
 * Concurrency: every call uses the same array, and its contents are whatever
 *   the last call left (the call clears what must start at zero); calls that
 *   overlap on the GPU (other streams, other threads) race and must be
 *   serialised by the caller.
 * The call synchronises `stream` (it reads the per-pixel arrays on the host)
 *   and returns EI_ERR_ARG for invalid arguments before it launches a kernel or
 *   writes device memory.
 */
#define EI_NOALLOC_SCRATCH_BYTES (32u << 20)
int ei_objective_grad_noalloc(const ei_geometry_desc *desc, const float *vol, const float *s_exp,
                              double *S_out, float *grad, void *stream);

/* Name and text of the last CUDA error this thread's library calls met (for
 * EI_ERR_CUDA / EI_ERR_ALLOC), or "" (thread-local storage). */
const char *ei_last_error(void);

/* Human-readable name of a status code (static storage). */
const char *ei_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* EI_H */
