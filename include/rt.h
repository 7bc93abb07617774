/*
 * rt.h -- C ABI of the GB300 bounce-map library.
 *
 * The library iterates the discrete bounce-to-bounce map of the intracavity
 * field E(x, y) of a high-Fresnel-number microchip laser (Okulov, "Two-
 * dimensional periodic and quasiperiodic spatial structures in microchip
 * laser resonator"): the nonlocal map of eq. conv_map written, as in the
 * integral-equation section (eqs. complex_8F, complex_aperture2), as a local
 * nonlinear gain step followed by the linear Fresnel propagator, the latter
 * applied in the Fourier basis as the operator exponent of eq.
 * limit_of_operators_renorm_final.  One bounce n -> n+1 computes
 *
 *   E'      = IDFT2( DFT2(E_n) * exp(-i pi alpha (mx^2 + my^2)) ) / n^2
 *   I       = |E'|^2
 *   E_{n+1} = sqrt(R) * A(x) A(y) * D(x, y) * exp(N_n / 2) * E'
 *   N_{n+1} = N_n + (N0(x, y) - N_n (1 + I / Isat)) / T1
 *
 * with alpha = (D/W)^2 / N_F (N_F = D^2 / (lambda z) the cavity Fresnel
 * number, D/W the gain-region diameter over the window width), A the hard
 * absorbing edge (0 on the outer edge_px pixels of each axis), N0 the pump
 * (unsaturated inversion) and (mx, my) the signed DFT frequencies.  Pixel j
 * sits at x_j = (j - n/2) / (n/2): the window half-width is 1.
 *
 * Multi-slice gain medium (opts.slices = m > 1; the thin-slice form of the
 * integral-equation section for a gain medium spread along the cavity):
 * a bounce is m steps "diffract z/m, then slice s", slice s amplifying
 * E <- exp(N_s / 2) E and relaxing N_s <- N_s + (N0/m - N_s (1 + I_s/Isat))/T1
 * with its own inversion N_s and the intensity I_s arriving at it; the
 * mirror (sqrt R, A, D) acts once, after the last slice.  m = 1 is the map
 * above.  The inversion of such a handle is m n x n arrays, slice-major, in
 * rt_read_inversion / rt_write_inversion; it starts at N0/m per slice.
 *
 * Aperture modulus.  A(j) = 0 on the outer edge_px pixels; with
 * taper_px = w > 0 it then rises over w pixels as sin^2((pi/2) (d+1)/(w+1)),
 * d = 0 .. w-1 the distance from the absorbing band, and is 1 inside
 * (a smooth, separable D_0 of eq. complex_aperture2).
 *
 * Inversion update.  RT_RELAX_EXACT replaces the explicit Euler step by the
 * exact solution of the rate equation dN/dt = (N0 - N (1 + I/Isat)) / T1 over
 * one bounce with I frozen: N <- Nss + (N - Nss) exp(-(1 + I/Isat)/T1),
 * Nss = N0 / (1 + I/Isat).  Both have the same fixed points.
 *
 * D is the phase of the complex aperture of eq. complex_aperture2 (a curved
 * mirror of focal length F and a random roughness phase psi):
 *
 *   D(x, y) = exp(-i (c (x^2 + y^2) + psi(x, y))),  c = (pi / (4 alpha)) (z / F),
 *
 * which is k r^2 / (2F) in window units (r = x W/2, k = 2 pi / lambda,
 * W^2 / lambda = z / alpha).  The paper prints exp(+i ...) together with the
 * opposite sign of the propagator (eq. Maxw_Bloch); the propagator above
 * follows eq. limit_of_operators_renorm_final, and the aperture phase is
 * conjugated with it, so the whole map is the complex conjugate of that
 * printed pair and F > 0 focuses (a concave mirror of radius of curvature
 * Rc has F = Rc / 2).  D = 1 unless z_over_F or roughness is set.
 *
 * Layout.  Grids are n x n, row-major (element [y*n + x]).  The field is
 * interleaved complex: complex64 (2 x float) for RT_FP32 handles, complex128
 * (2 x double) for RT_FP64 handles.  The inversion is float or double alike.
 *
 * Ownership.  The library owns every device buffer it allocates; the caller
 * owns every pointer it passes in and keeps it valid for the duration of the
 * call.  Pointers marked "host or device" may point to either (unified
 * addressing decides the copy direction).
 *
 * Errors.  Every call returns an rt_status; none aborts the process.  A
 * device-side error (non-finite intensity) is sticky: it is reported by the
 * next call that synchronises (rt_sync, rt_read_*, rt_stats).
 *
 * Threading.  A handle is not thread-safe; distinct handles may be used from
 * distinct threads.  All work of a handle is ordered on its stream.
 */
#ifndef RT_H
#define RT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_handle rt_handle;

typedef enum {
    RT_OK = 0,
    RT_EINVAL = -1,    /* bad argument: size, range, null pointer, byte count */
    RT_ENOMEM = -2,    /* device or host allocation failed */
    RT_ECUDA = -3,     /* a CUDA runtime call failed */
    RT_ENUMERIC = -4,  /* the field's mean intensity became NaN or Inf */
    RT_ETIMEOUT = -5,  /* a bounded wait ran out */
    RT_EBUSY = -6,     /* the handle or server cannot take the request now */
    RT_EBOUNDS = -7,   /* an index left its buffer (bounds-checked builds only; the access was skipped) */
    RT_ECANCELED = -8  /* a served request was cancelled (rt_serve_cancel) */
} rt_status;

enum { RT_PUMP_SUPERGAUSS = 0, RT_PUMP_UNIFORM = 1, RT_PUMP_ARRAY = 2 };
enum { RT_FP32 = 0, RT_FP64 = 1 };
enum { RT_RELAX_EULER = 0, RT_RELAX_EXACT = 1 };

/* Pump, i.e. the unsaturated inversion N0 = g0 * P(x, y):
 *   RT_PUMP_SUPERGAUSS  P = exp(-(r / radius)^order), r = sqrt(x^2 + y^2),
 *                       radius as a fraction of the window half-width;
 *   RT_PUMP_UNIFORM     P = 1;
 *   RT_PUMP_ARRAY       P = profile[y*n + x] (host array of n*n doubles,
 *                       copied at creation).
 * A NULL pump means super-Gaussian, order 10, radius 0.8. */
typedef struct {
    int kind;
    double order;
    double radius;
    const double *profile;
} rt_pump;

/* Options; rt_opts_default fills the defaults listed per field. */
typedef struct {
    double Isat;                  /* saturation intensity (1) */
    int edge_px;                  /* absorbing edge width in pixels (8) */
    int precision;                /* RT_FP32 (fused FP32 path) or RT_FP64 (plain FP64 path) */
    unsigned long long seed;      /* noise seed (14102855) */
    double noise_amp;             /* initial noise amplitude, E|E|^2 = amp^2 (1e-6) */
    double pump_diam_over_window; /* D/W in alpha = (D/W)^2 / N_F (0.8) */
    void *cuda_stream;            /* cudaStream_t to run on; NULL = the legacy default stream */
    long long history_cap;        /* >0: keep the mean intensity of the last history_cap bounces (65536) */
    int chunk;                    /* bounces per captured CUDA graph in rt_step; 0 = no graphs (500) */
    int col_tile;                 /* FP32 column-sweep tile width in columns (2, 4, 8 or 16); 0 = library choice (0) */
    double z_over_F;              /* curved mirror: propagation distance per bounce over its focal length F,
                                     > 0 focuses, 0 = flat mirror (0); finite */
    const double *roughness;      /* mirror roughness: host array of n*n doubles psi[y*n + x] in radians,
                                     copied at creation; NULL = smooth (NULL) */
    int slices;                   /* gain medium as m thin slices per bounce, 1 <= m <= 64 (0 or 1: one
                                     slice at the mirror; handles only, see below) (0) */
    int taper_px;                 /* smooth aperture: width in pixels of the sin^2 ramp inside the
                                     absorbing edge, 0 = hard edge (0) */
    int relax;                    /* inversion update: RT_RELAX_EULER (the map above) or RT_RELAX_EXACT
                                     (the rate equation solved over the bounce, see below) (EULER) */
} rt_opts;

rt_status rt_opts_default(rt_opts *opts);

/* Statistics of a handle (rt_stats). */
typedef struct {
    long long bounces;        /* bounces completed since creation */
    double mean_intensity;    /* <|E|^2> after the last bounce (FP64 accumulation); 0 before any bounce */
    double alpha;             /* lambda z / W^2 in use */
    int n;                    /* grid side */
    int precision;            /* RT_FP32 or RT_FP64 */
    int last_error;           /* sticky device error as an rt_status (RT_OK if none) */
    long long history_len;    /* bounces currently held in the history ring */
} rt_stats_t;

/* Create a resonator of side n (power of two, 32 <= n <= 4096) with Fresnel
 * number `fresnel` (> 0), pump `pump`, small-signal gain g0 (intensity gain
 * exponent per pass, >= 0), inversion relaxation time T1 (in bounces, >= 1)
 * and mirror reflectivity R (0 < R <= 1).  Allocates the field, inversion and
 * tables on the device, draws the seeded complex Gaussian noise field
 * (splitmix64 counter stream + Box-Muller, in FP64, rounded to the handle's
 * precision) and sets N = N0 (N0/m per slice).  Section "Integral equation form", eqs.
 * complex_8F and complex_aperture2; the noise start and the full inversion
 * are the initial condition of the map.
 * Returns RT_EINVAL for out-of-range arguments, RT_ENOMEM, RT_ECUDA. */
rt_status rt_create(int n, double fresnel, const rt_pump *pump, double g0, double T1, double R,
                    const rt_opts *opts, rt_handle **out);

/* Enqueue n_bounces (>= 0) iterations of the map on the handle's stream and
 * return without waiting.  Eq. conv_map / complex_8F per bounce, the
 * propagator of eq. limit_of_operators_renorm_final. */
rt_status rt_step(rt_handle *h, long long n_bounces);

/* One half of a bounce, for per-kernel timing: RT_SWEEP_COLUMNS enqueues the
 * column sweep (1-D diffraction along y of every column), RT_SWEEP_ROWS the
 * row sweep (1-D diffraction along x of every row, then the local map:
 * gain, mirror, edge, inversion update, mean intensity).  A bounce is the
 * column sweep followed by the row sweep, which is exactly what rt_step
 * enqueues; the propagator factorisation follows from eq.
 * limit_of_operators_renorm_final with a separable Laplacian.  Calling the
 * row sweep without the column sweep first is not a bounce of the map.
 * FP32 single-slice handles only (RT_EINVAL otherwise).  Asynchronous. */
enum { RT_SWEEP_COLUMNS = 0, RT_SWEEP_ROWS = 1 };
rt_status rt_sweep(rt_handle *h, int which);

/* Wait for the handle's stream; reports a sticky device error.
 * Infrastructure (no counterpart in the paper). */
rt_status rt_sync(rt_handle *h);

/* Copy the current field (n*n complex64 or complex128, `bytes` must equal
 * n*n*8 or n*n*16) to dst (host or device).  Blocks until the copy is done.
 * The field is E_n of eq. conv_map, the state of the map at the mirror and
 * gain plane after the last bounce. */
rt_status rt_read_field(rt_handle *h, void *dst, size_t bytes);

/* Copy the current inversion (n*n float or double) to dst (host or device).
 * Blocks.  The inversion is N_n, the second state variable of eq. conv_map
 * (relaxed as the rate equation of eq. Maxw_Bloch_incoherent). */
rt_status rt_read_inversion(rt_handle *h, void *dst, size_t bytes);

/* Replace the field / inversion with src (host or device, same layouts as
 * the reads): checkpoint restore or a caller-chosen initial condition.
 * Ordered on the handle's stream; src must stay valid until rt_sync.
 * Infrastructure (the paper starts every run from noise). */
rt_status rt_write_field(rt_handle *h, const void *src, size_t bytes);
rt_status rt_write_inversion(rt_handle *h, const void *src, size_t bytes);

/* Set the bounce counter (used when restoring a checkpoint).  Infrastructure. */
rt_status rt_set_bounces(rt_handle *h, long long bounces);

/* Synchronise and report counters (bounce count, last mean intensity
 * <|E_n|^2>, the sticky error).  Infrastructure: a diagnostic of the map. */
rt_status rt_stats(rt_handle *h, rt_stats_t *out);

/* Copy the mean intensity <|E|^2> of the most recent bounces, oldest first,
 * into dst (host, up to max values); *got receives the count written.
 * Infrastructure: the intensity history of the iterates n of eq. conv_map. */
rt_status rt_read_history(rt_handle *h, double *dst, long long max, long long *got);

/* Far-field spectrum S = |DFT2(E)|^2 of the current field (n*n float or
 * double, unnormalised) to dst (host or device).  Blocks.  The Fourier image
 * of the field that the multiscale section describes (its period p_m at the
 * planes L_m); the DFT is the Fourier basis of eq.
 * limit_of_operators_renorm_final. */
rt_status rt_read_spectrum(rt_handle *h, void *dst, size_t bytes);

/* Structured starting fields of the exact solutions (section "Exact
 * solutions", eqs. Field_exact11 and Field_exact112), evaluated in FP64 on
 * the periodic window (x, y in [-1, 1), period 2):
 *
 *   E = amplitude * exp(-r^2 / (2 envelope^2)) * exp(-i curvature r^2) * S,
 *
 * envelope 0 meaning no envelope, and S
 *   RT_PATTERN_GAUSSIAN      exp(-r^2 / (2 width^2)), one beam on the axis;
 *   RT_PATTERN_BEAM_ARRAY    sum over the periods^2 lattice points (a p, b p),
 *                            p = 2 / periods, a, b = 0 .. periods-1, of
 *                            s_ab exp(-d^2 / (2 width^2));
 *   RT_PATTERN_VORTEX_ARRAY  the same sum of first-order vortices
 *                            ((dx + i k_ab dy) / width) exp(-d^2 / (2 width^2)),
 * with (dx, dy) the shortest displacement from the lattice point on the
 * periodic window, d^2 = dx^2 + dy^2, terms with d^2 / (2 width^2) > 50
 * left out, and s_ab (beam sign) or k_ab (vortex charge) = (-1)^(a+b) when
 * out_of_phase is set (periods must then be even), else 1.
 * The Talbot condition of eq. Field_exact11 (cavity length m p^2 / lambda)
 * is alpha * periods^2 = 2m in the units of this library. */
enum { RT_PATTERN_GAUSSIAN = 0, RT_PATTERN_BEAM_ARRAY = 1, RT_PATTERN_VORTEX_ARRAY = 2 };
typedef struct {
    int kind;             /* RT_PATTERN_* */
    int periods;          /* arrays: lattice periods across the window (>= 1) */
    int out_of_phase;     /* arrays: neighbours alternate in sign (beams) or charge (vortices) */
    double width;         /* beam or vortex-core radius, window units (> 0) */
    double envelope;      /* radius of the common Gaussian envelope (>= 0; 0 = none) */
    double curvature;     /* common phase front exp(-i curvature r^2) (finite) */
    double amplitude;     /* overall factor (finite) */
} rt_pattern;

/* Replace the handle's field with a structured field (ordered on the
 * handle's stream; the inversion and counters are left as they are).
 * RT_EINVAL for an invalid pattern. */
rt_status rt_set_field_pattern(rt_handle *h, const rt_pattern *pattern);

/* The field at an intracavity plane: the current field (at the mirror and
 * gain plane) diffracted a further zeta * z, zeta any finite real (negative
 * values propagate backwards; zeta = 1 is one bounce's diffraction without
 * the local map):
 *   E_zeta = IDFT2( DFT2(E) * exp(-i pi alpha zeta (mx^2 + my^2)) ) / n^2.
 * The planes L_m = p^2 / (2 lambda m) between the mirrors, where the arrays
 * of period p/m form (section "Comparison with experiment"), are
 * zeta = L_m / z.  Written to dst (host or device) in the layout of
 * rt_read_field; the handle's state is unchanged.  Blocks. */
rt_status rt_read_field_at(rt_handle *h, double zeta, void *dst, size_t bytes);

/* Dominant spatial frequency of the current field.  Bin k and its mirror
 * -k (mod n) form one peak of folded power S[k] + S[-k] (S[k] once if
 * k == -k), filed under the smaller row-major index; with ring > 0 only
 * bins with max(|mx|, |my|) >= ring compete; ties go to the smaller index.
 * Writes the signed (mx, my) and the folded power. Blocks. */
rt_status rt_spectrum_peak(rt_handle *h, int ring, int *mx, int *my, double *power);

/* ---- autotuning ---------------------------------------------------------
 * The column sweep's tile width (columns per block: 2, 4, 8 or 16) trades
 * load balance and copy-engine box width against shared memory and
 * occupancy, and its radix order decides where the one pass of radix 2, 4
 * or 8 goes when 4 does not divide log2 n (order 0: after the radix-16
 * passes; 1: first; 2: second, after one radix-16 pass), which changes the
 * exchange and twiddle pattern.  rt_autotune times the column sweep of a
 * scratch n x n field on the current device for every width that fits and
 * every order (reps launches each, CUDA events) and records the fastest pair
 * for this process; handles, batches and servers created afterwards with
 * col_tile = 0 use both (per-class batch launches; mixed launches use order
 * 0), so a batch slot or a served request gives the bits of a handle.  rt_tune_set / rt_tune_set_order
 * record a width or an order directly (e.g. loaded from a JSON cache file by
 * the Python binding); rt_tune_get reports the width in use for n (tuned,
 * or the built-in default; *tuned says which) and rt_tune_get_order the
 * order and the number of orders n offers.  Every order computes the same
 * DFT; the roundings differ.  Not part of the paper's method. */
rt_status rt_autotune(int n, int reps, int *best_col_tile, double *best_us);
/* The same choice made for the work as it runs: `resonators` (1..16) n x n
 * FP32 handles (N_F 1000, default pump, g0 0.3, T1 1e4, R 0.9), each on a
 * stream of its own with one CUDA graph per `bounces` (1..1e5) bounces, are
 * stepped together for every width that fits and every order; the pair with
 * the highest rate (best of `reps` >= 1 timings, host clock around the steps
 * and the waits) is recorded as rt_autotune records its pair, and written to
 * *best_col_tile, *best_order and *best_rate (round trips/s over all the
 * resonators).  A column sweep timed alone and the same sweep sharing the
 * GPU with other resonators' sweeps can favour different pairs (a wider tile
 * holds more shared memory per block, which the concurrent sweeps then
 * cannot use).  Allocates and frees the handles' memory; blocks.  While it
 * runs, the process-wide choice for side n goes through every candidate, so
 * handles, batches or servers created meanwhile by other threads may take
 * one of them (any pair gives results within the same tolerances).
 * RT_EINVAL for arguments out of range; on a failure the earlier choice
 * stays. */
rt_status rt_autotune_concurrent(int n, int resonators, int bounces, int reps, int *best_col_tile, int *best_order,
                                 double *best_rate);
rt_status rt_tune_set(int n, int col_tile);
rt_status rt_tune_get(int n, int *col_tile, int *tuned);
rt_status rt_tune_set_order(int n, int order);
rt_status rt_tune_get_order(int n, int *order, int *orders);

/* Launch form of batches and servers created afterwards.  mixed = 1:
 * resonators of sides 128..2048 share one persistent launch per sweep
 * whatever their sizes; every work item holds the same number of points
 * (column tiles of 8192/n columns, row groups of 2048/n rows) and is
 * dispatched on its grid size inside the launch, so the classes fill one
 * another's tails (a batch's graph may split the resonators into several
 * such launches, one per graph chain: rt_tune_set_batch_split).  mixed = 0
 * (the default): one launch per sweep and size class, column tiles of the
 * tuned width, one or more graph chains per class.
 * Batches created with a nonzero col_tile always use per-class launches.
 * The fields are the same either way; the Python binding's
 * tune.autotune_batch times both on a batch and keeps the faster. */
rt_status rt_tune_set_batch_mixed(int mixed);
rt_status rt_tune_get_batch_mixed(int *mixed);
/* Graph branches of batches: a batch's graph of `chunk` bounces runs each
 * size class (or, in the mixed form, the mixed launches) as `parts` chains
 * of consecutive resonators on streams of their own, which overlap one
 * another's phases and tails.  parts = 0 (the default) takes ceil(3 / c)
 * parts for c chains at one part each, about three chains in all; 1..8 sets
 * the parts per class for graphs captured from now on (the fields do not
 * depend on it).  The Python binding's tune.autotune_batch times the launch
 * forms with 1..4 parts and keeps the fastest.  RT_EINVAL outside 0..8. */
rt_status rt_tune_set_batch_split(int parts);
rt_status rt_tune_get_batch_split(int *parts);

/* ---- batches of resonators ---------------------------------------------
 * Many independent resonators (eq. conv_map per resonator, each with its
 * own grid size, Fresnel number, pump, gain, T1, R) stepped together: the
 * resonators of one grid size share each persistent launch of the two
 * sweeps, so small grids fill the GPU and large batches keep every SM busy.
 * FP32 only; 32 <= n <= 2048 per job. */
typedef struct {
    int n;                        /* grid side (power of two, 32..2048) */
    double fresnel;               /* N_F */
    double g0, T1, R;             /* gain exponent per pass, relaxation (bounces), mirror reflectivity */
    rt_pump pump;                 /* pump (profile copied at set-up) */
    double Isat;                  /* saturation intensity */
    int edge_px;                  /* absorbing edge width */
    unsigned long long seed;      /* noise seed */
    double noise_amp;             /* noise amplitude */
    double pump_diam_over_window; /* D/W */
    double z_over_F;              /* curved mirror z / F (0 = flat) */
    const double *roughness;      /* n*n roughness phase psi, host, copied at set-up; NULL = smooth */
    int taper_px;                 /* smooth aperture ramp width (0 = hard edge) */
    int relax;                    /* RT_RELAX_EULER or RT_RELAX_EXACT */
} rt_job;

/* Fill a job with the defaults of rt_opts_default / rt_create for side n. */
rt_status rt_job_default(rt_job *job, int n);

typedef struct rt_batch rt_batch;

/* Create a batch of `count` resonators (slots 0..count-1) from jobs.
 * opts: cuda_stream, history_cap, chunk and col_tile are used; precision
 * must be RT_FP32.  Every slot starts as rt_create would start it and runs
 * without a bounce limit.  RT_EINVAL, RT_ENOMEM, RT_ECUDA. */
rt_status rt_batch_create(const rt_job *jobs, int count, const rt_opts *opts, rt_batch **out);

/* Enqueue n_bounces iterations for every slot that has bounces left.  Async. */
rt_status rt_batch_step(rt_batch *b, long long n_bounces);

/* One half of a bounce over every active slot, for per-kernel timing:
 * RT_SWEEP_COLUMNS or RT_SWEEP_ROWS (see rt_sweep).  Async. */
rt_status rt_batch_sweep(rt_batch *b, int which);

/* Re-initialise slot i with a new job of the same n (fresh noise field,
 * N = N0, counters at zero).  The slot then runs n_bounces more bounces and
 * stops (n_bounces < 0: no limit; 0: the slot stays idle).  Ordered on the
 * batch stream.  Used by the serving loop to recycle slots. */
rt_status rt_batch_set_job(rt_batch *b, int i, const rt_job *job, long long n_bounces);

/* Wait for the batch stream; reports a sticky device error of any slot. */
rt_status rt_batch_sync(rt_batch *b);

/* Per-slot copies, layouts as rt_read_field etc.  Reads block. */
rt_status rt_batch_read_field(rt_batch *b, int i, void *dst, size_t bytes);
rt_status rt_batch_read_inversion(rt_batch *b, int i, void *dst, size_t bytes);
rt_status rt_batch_write_field(rt_batch *b, int i, const void *src, size_t bytes);
rt_status rt_batch_write_inversion(rt_batch *b, int i, const void *src, size_t bytes);

/* Per-slot counters (synchronises). */
rt_status rt_batch_stats(rt_batch *b, int i, rt_stats_t *out);

/* Mean intensity of slot i's most recent bounces, oldest first (host dst). */
rt_status rt_batch_read_history(rt_batch *b, int i, double *dst, long long max, long long *got);

/* Bounce counters of all slots into counts[count] (host; synchronises). */
rt_status rt_batch_bounces(rt_batch *b, long long *counts);

/* Device bytes held by the batch. */
rt_status rt_batch_footprint(rt_batch *b, size_t *bytes);

rt_status rt_batch_destroy(rt_batch *b);

/* ---- serving: continuous batching of simulation requests -----------------
 * A server owns one GPU stream and a device-memory budget.  Requests (a job
 * and a bounce count) may be submitted at any time from any thread.  A
 * worker thread runs scheduling rounds: it admits queued requests (oldest
 * first) while their footprint fits the budget, runs `chunk` bounces of
 * every resident request in shared batched launches (requests of one grid
 * size share each launch; a request stops exactly at its own bounce count),
 * then retires finished requests, copying each final field to the buffer
 * given at submission.  State stays on the device between rounds.  A
 * request's result is the same as running it alone on a handle.  A request
 * whose set-up fails waits for room while others run; if it still cannot be
 * placed with nothing else resident (every idle slot released), its result
 * is posted at once with RT_ENOMEM (allocation failed) or RT_ECUDA. */
typedef struct rt_server rt_server;

enum { RT_SERVE_FIFO = 0, RT_SERVE_SHORTEST_FIRST = 1 };

typedef struct {
    long long budget_bytes;   /* device memory for resident requests (8 GiB) */
    int chunk;                /* bounces per scheduling round (500) */
    int max_per_size;         /* resident requests of one grid size at most (128) */
    void *cuda_stream;        /* stream to run on; NULL = the server creates its own */
    int policy;               /* RT_SERVE_FIFO: every resident request advances chunk bounces per round;
                                 RT_SERVE_SHORTEST_FIRST: each round advances only the resident requests
                                 with the least remaining work (n^2 x bounces left, ties by submission)
                                 until their points reach round_points; the others wait (FIFO) */
    long long round_points;   /* shortest-first: grid points advanced per round (0 = 2^23, two 2048^2 grids) */
} rt_serve_opts;

typedef struct {
    long long id;             /* from rt_serve_submit */
    int status;               /* RT_OK, or the error that ended the request (RT_ECANCELED, RT_ENOMEM, ...) */
    int n;                    /* grid side */
    long long bounces;        /* bounces run */
    double mean_intensity;    /* <|E|^2> after the last bounce */
    double submit_s;          /* server clock (seconds since creation): submission */
    double admit_s;           /* admission (first round that ran it) */
    double finish_s;          /* completion (its field copied out) */
} rt_result;

typedef struct {
    long long submitted, queued, running, done;
    long long resident_bytes;          /* device bytes held for requests */
    double point_bounces;              /* sum over finished rounds of n^2 x bounces run */
    double busy_s;                     /* wall time spent in scheduling rounds */
    long long rounds;
    long long peak_resident_bytes;     /* most device bytes ever held for requests at once (<= budget) */
} rt_serve_stats_t;

rt_status rt_serve_opts_default(rt_serve_opts *opts);
rt_status rt_serve_create(const rt_serve_opts *opts, rt_server **out);

/* Queue a request of n_bounces (> 0) bounces of `job` (32 <= n <= 2048,
 * super-Gaussian order-10 or uniform pump, flat or curved mirror without a
 * roughness table).  field_out (host or device, n*n complex64, may be NULL)
 * receives the final field before the result is posted; it must stay valid
 * until then.  *id receives the request id.
 * RT_EINVAL for bad jobs or a request that could never fit the budget. */
rt_status rt_serve_submit(rt_server *s, const rt_job *job, long long n_bounces, void *field_out, long long *id);

/* Cancel request `id`: a queued request is dropped at once, a running one
 * stops after the current scheduling round; either way its result is posted
 * with status RT_ECANCELED, the bounces it ran, and field_out left
 * unwritten.  RT_EINVAL if the id is unknown or its result was already
 * posted. */
rt_status rt_serve_cancel(rt_server *s, long long id);

/* Move up to `max` finished results into out (oldest first); *got = count. */
rt_status rt_serve_poll(rt_server *s, rt_result *out, int max, int *got);

/* Wait until every submitted request has finished or `timeout_s` passes
 * (RT_ETIMEOUT). */
rt_status rt_serve_drain(rt_server *s, double timeout_s);

rt_status rt_serve_stats(rt_server *s, rt_serve_stats_t *out);

/* Stop the worker (queued requests are dropped) and free everything. */
rt_status rt_serve_destroy(rt_server *s);

/* ---- allocation-free stepping ------------------------------------------
 * The paper has no counterpart to this entry point.  It exists for callers
 * that cannot call cudaMalloc: a host that hands the library device buffers
 * from its own memory pool or fixed budget and forbids any other device
 * allocation (a plugin inside a framework that owns all device memory), or a
 * latency-critical loop in which an allocation could synchronise the device
 * and stall.
 *
 * rt_step_noalloc runs n_bounces of the fused FP32 bounce (the kernels that
 * rt_step runs on an RT_FP32 handle) directly on the caller's device
 * buffers, updated in place: `field` (n*n complex64, row-major) and
 * `inversion` (n*n float), both 16-byte aligned.  It allocates nothing.  The
 * scratch it needs (propagator and twiddle tables, reduction partials,
 * counters) lives in one fixed array of about 130 KB of device memory that
 * every GPU which loads this library holds until the process exits; n is
 * therefore limited to RT_NOALLOC_MAX_N, and larger sizes return RT_EINVAL.
 * Supported: RT_FP32 only, super-Gaussian pump of order 10 or uniform pump,
 * flat or curved mirror without roughness (anything else returns
 * RT_EINVAL).  Options used: Isat, edge_px, pump_diam_over_window,
 * cuda_stream, col_tile, z_over_F, taper_px, relax (NULL opts = defaults).
 *
 * The first call in each CUDA context (per device, and again after
 * cudaDeviceReset) looks up the array's device address with that device
 * current; make that first call before any stream capture.
 * All calls share the one array: each call rebuilds the tables and clears
 * the counters it needs, and calls whose work overlaps on the GPU race with
 * one another, so order them on one stream or with events.
 * With mean_intensity == NULL the call is asynchronous on the stream.  With
 * a host pointer it waits for the work, stores <|E|^2> after the last
 * bounce, and returns a device error (RT_ENUMERIC, RT_ETIMEOUT) if one
 * occurred in this call or in an asynchronous call before it: such an error
 * stays in the array until a synchronous call reports it, once. */
#define RT_NOALLOC_MAX_N 4096
rt_status rt_step_noalloc(int n, double fresnel, const rt_pump *pump, double g0, double T1, double R,
                          const rt_opts *opts, void *field, void *inversion, long long n_bounces,
                          double *mean_intensity);

/* ---- test hook -----------------------------------------------------------
 * Fault injection for tests of the out-of-memory paths (not part of the
 * method): the after-th device allocation the library makes from now on
 * (0 = the next one) fails once as if the device were out of memory; a
 * negative value cancels a pending failure.  The failure is produced on the
 * host before any device call.  Process-wide; returns RT_OK. */
rt_status rt_debug_fail_alloc(int after);
/* The same for `count` consecutive allocations starting with the after-th
 * (count < 0: every one from the after-th on, until cancelled by a negative
 * `after`).  rt_debug_fail_alloc(a) is rt_debug_fail_alloc_n(a, 1). */
rt_status rt_debug_fail_alloc_n(int after, int count);
/* Test of the sweeps' bounded copy waits: one block arms a stage barrier
 * for a copy that is never issued (with drain != 0 also the second stage,
 * as if the next item's copy were in flight) and runs the sweeps' own stage
 * wait, which gives up after its limit (about 2 s; twice that with drain)
 * with nothing left in flight.  *device_status receives the block's error
 * word (RT_ETIMEOUT expected).  Returns RT_OK once the probe has ended,
 * RT_ENOMEM or RT_ECUDA on a host-side failure, RT_EINVAL for NULL. */
rt_status rt_debug_wait_probe(int drain, int *device_status);

/* Release every device buffer and graph of the handle (NULL is accepted).
 * Infrastructure. */
rt_status rt_destroy(rt_handle *h);

/* Static, human-readable name of a status code.  Infrastructure. */
const char *rt_status_string(rt_status s);

/* Library version (major * 10000 + minor * 100 + patch).  Infrastructure. */
int rt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RT_H */
