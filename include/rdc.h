/*
 * rdc.h -- C ABI of librdc, a GPU (sm_103a) time-stepper for the
 * two-variable Oregonator reaction-diffusion model.
 *
 * The model (Eq. 1, §2 of "RDCSim: a GPU-Accelerated, Interactive Simulator
 * for Reaction-Diffusion Chemistry"):
 *
 *     u_t = (1/eps) [ u - u^2 - (f v + phi(x,y)) (u - q)/(u + q) ] + Du lap(u)
 *     v_t = u - v
 *
 * integrated with explicit forward Euler (timestep dt) and the five-node
 * discrete Laplacian on a square grid of spacing dx (§2, the paragraph after
 * Table 1); phi is a per-cell excitability map (§2, §3: active and passive
 * substrate).  Defaults are Table 1.  Catalytic stimulation sets u of the
 * stimulated cells to a value (§2).
 *
 * Points the paper leaves open are fixed as follows, and every kernel
 * behind this header follows them:
 *   - zero-flux borders: a neighbour outside the grid takes the value of
 *     the border cell itself (cell-centred mirror);
 *   - Jacobi update: u' and v' are both computed from step n;
 *   - initial state: u = v = u*(phi) per cell, the homogeneous rest state;
 *   - Laplacian summed as ((w + e) + (n + s)) - 4 c, scaled by 1/(dx*dx);
 *   - no clamping of u or v.
 *
 * Conventions for every call:
 *   - Each call returns an int status (RDC_OK = 0 on success).  Invalid
 *     arguments return RDC_EINVAL and change nothing.
 *   - Grids are H rows by W columns, row-major; cell (i, j) is row i (y),
 *     column j (x); host arrays are packed (row stride W elements).
 *   - Host input buffers are copied before the call returns; the caller
 *     owns all host buffers.  Device memory belongs to the library except
 *     with rdc_create_ext, where the caller owns it and must keep it alive
 *     until rdc_destroy.
 *   - All device work of a simulation runs on its CUDA stream, in call
 *     order.  Calls marked "async" only enqueue work; calls that return
 *     host data synchronise that stream.
 *   - A handle is not thread-safe; distinct handles may be used from
 *     distinct threads.
 */
#ifndef RDC_H_
#define RDC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RDC_OK 0
#define RDC_EINVAL 1          /* invalid argument; nothing was changed */
#define RDC_ENOMEM 2          /* a device or host allocation failed */
#define RDC_ECUDA 3           /* a CUDA call failed (message: rdc_last_error) */
#define RDC_ENONFINITE 4      /* the state holds a non-finite u or u + q <= 0 */
#define RDC_ETIMEOUT 5        /* a bounded device wait gave up */
#define RDC_EUNSTABLE_WARN 6  /* informational: forward Euler is linearly
                                 unstable at the rest state of some phi */
#define RDC_EUNSUPPORTED 7    /* valid request this build cannot serve */

/* ---- precision modes ---------------------------------------------------- */
/* Arithmetic and storage of u, v (and phi) on the device. */
#define RDC_F32 0             /* FP32 compute, FP32 u/v/phi (20 B per cell-update) */
#define RDC_F64 1             /* FP64 compute and storage; op order identical to
                                 the sequence documented at rdc_step, with no
                                 contraction, so results are bit-reproducible
                                 against any IEEE FP64 implementation of it */
#define RDC_F32_BF16STORE 2   /* FP32 compute, u/v stored as bfloat16 (RN-even),
                                 phi FP32 (12 B per cell-update) */
#define RDC_F32_F16STORE 3    /* FP32 compute, u/v stored as IEEE half (RN-even),
                                 phi FP32 */

/* ---- host buffer element types ------------------------------------------ */
#define RDC_DTYPE_F32 0
#define RDC_DTYPE_F64 1
#define RDC_DTYPE_BF16 2
#define RDC_DTYPE_F16 3

/* ---- flags (0 = the full model, rounded to nearest) ---------------------- */
#define RDC_DIFFUSION_ONLY 1  /* test mode: drop the reaction term from u_t */
#define RDC_REACTION_ONLY 2   /* test mode: drop Du lap(u) from u_t */
/*
 * Stochastic rounding (16-bit storage only: RDC_F32_BF16STORE,
 * RDC_F32_F16STORE).  Each new u', v' (an FP32 value x) is rounded to the
 * storage type at random instead of to nearest: with lo = x rounded toward
 * zero and hi the next storage value away from zero, the result is hi when
 *     r16 < 2^16 (|x| - |lo|) / (|hi| - |lo|)
 * and lo otherwise, r16 being 16 random bits (non-finite x, and FP16 beyond
 * 65504, round to nearest).  The expected stored value is then x, so small
 * per-step increments (dt (u - v) is often below half a BF16 spacing of v)
 * survive on average instead of being lost every step.  The random bits
 * come from Philox4x32-10 (Salmon et al., SC'11) with counter
 * (column / 4, row, step index mod 2^32, step index / 2^32) and key
 * (round_seed, 0): word (column mod 4) of the output, whose top 16 bits are
 * r16 for the cell's u and whose low 16 bits are r16 for its v.  The step
 * index is the index of the state being written (steps since rdc_create or
 * rdc_reset_rest).
 * Results are deterministic and identical for every k_block, launch shape
 * and batch; rdc_stoch_round_sample exposes the rounding.  Not available in
 * rdc_step_noalloc.
 */
#define RDC_STOCH_ROUND 4

typedef struct rdc_sim rdc_sim; /* opaque simulation handle */

typedef struct {
    int32_t width;   /* W, columns (x), >= 1 */
    int32_t height;  /* H, rows (y), >= 1 */
} rdc_grid;

/* Model and run parameters.  rdc_params_default fills Table 1. */
typedef struct {
    double eps;        /* epsilon, time-scale ratio            (Table 1: 0.0243) */
    double f;          /* stoichiometric factor                (Table 1: 1.4)    */
    double q;          /* propagation scaling factor           (Table 1: 0.002)  */
    double Du;         /* diffusion coefficient of u           (Table 1: 0.45)   */
    double dt;         /* Euler timestep                       (Table 1: 0.001)  */
    double dx;         /* grid spacing                         (Table 1: 0.25)   */
    int32_t precision; /* RDC_F32 / RDC_F64 / RDC_F32_BF16STORE / RDC_F32_F16STORE */
    int32_t flags;     /* RDC_DIFFUSION_ONLY | RDC_REACTION_ONLY (not both),
                          | RDC_STOCH_ROUND */
    int32_t k_block;   /* Euler steps fused per launch (temporal blocking):
                          0 = library default (4 for FP32-compute grids of
                          >= 2^20 cells in the full model, else 1; see
                          rdc_tune),
                          1 = one step per launch,
                          2..8 = k steps per launch.  Results are bitwise
                          identical for every k. */
    int32_t round_seed; /* key of the stochastic rounding stream (used as an
                           unsigned 32-bit value); must be 0 without
                           RDC_STOCH_ROUND */
} rdc_params;

/* Fills *out with Table 1 (eps, f, q, Du, dt, dx), RDC_F32, flags 0,
 * k_block 0.  Returns RDC_EINVAL if out is NULL. */
int rdc_params_default(rdc_params* out);

/*
 * Creates a simulation of grid g and sets it to the rest state
 * u = v = u*(phi) of every cell (see rdc_rest_state).
 *   phi_host : H*W floats, row-major, copied; NULL = uniform phi_active
 *              (Table 1: 0.054).  Each value must be finite and exceed
 *              q (1 + f) so that a positive rest state exists.
 *   stream   : a cudaStream_t to run on (cudaStreamLegacy and
 *              cudaStreamPerThread are accepted), or NULL for a
 *              library-owned non-blocking stream.  A caller's stream must
 *              outlive the simulation.
 *   out      : receives the handle; *out is NULL on failure.
 * The call also records whether forward Euler is linearly unstable at the
 * rest state of the map's largest phi (as rdc_stability computes it; phi =
 * 0.2, the workloads' passive background, is): rdc_view's unstable and
 * stability_rho hold the result, kept current by every call that changes
 * phi.  rdc_create still returns RDC_OK then; the handle is usable.
 * Validation (RDC_EINVAL): W or H < 1; a non-finite parameter; eps, q, dt
 * or dx <= 0; Du < 0; f + q <= 1; Du dt / dx^2 > 1/4 (the explicit
 * diffusion limit); both test flags set; RDC_STOCH_ROUND with FP32 or FP64
 * storage; an unknown flag; k_block outside 0..8; round_seed != 0 without
 * RDC_STOCH_ROUND.
 * The device must be sm_103 (RDC_EUNSUPPORTED otherwise).
 */
int rdc_create(rdc_grid g, const rdc_params* p, const float* phi_host,
               void* stream, rdc_sim** out);

/* As rdc_create with a double-precision phi map (for RDC_F64 parity runs;
 * in FP32 modes the values are rounded to float). */
int rdc_create_f64phi(rdc_grid g, const rdc_params* p, const double* phi_host,
                      void* stream, rdc_sim** out);

/*
 * As rdc_create, on caller-owned device memory (for example torch tensors).
 *   dev_u[2], dev_v[2] : two state buffers each (ping-pong), storage type of
 *                        p->precision, row pitch pitch_bytes;
 *   dev_phi            : phi map, float (double for RDC_F64), same pitch in
 *                        elements as the state planes: pitch_bytes / sizeof
 *                        of the state element;
 *   pitch_bytes        : a multiple of 16 bytes, >= W * element size.
 * All pointers must be 16-byte aligned.  The state is NOT initialised: the
 * current state is dev_u[0], dev_v[0] as the caller left it (use
 * rdc_reset_rest to set the rest state).  The library never frees them.
 * The map's largest value (for the stability record) is found on the device;
 * the call synchronises the stream.
 */
int rdc_create_ext(rdc_grid g, const rdc_params* p, void* const dev_u[2],
                   void* const dev_v[2], const void* dev_phi,
                   size_t pitch_bytes, void* stream, rdc_sim** out);

/* Destroys the handle and frees library-owned memory; waits for the
 * simulation's stream first.  NULL is a no-op. */
void rdc_destroy(rdc_sim* sim);

/* Async.  Replaces the phi map (host, H*W of dtype RDC_DTYPE_F32 or
 * RDC_DTYPE_F64) and resets the state to the rest state of the new map. */
int rdc_set_phi(rdc_sim* sim, const void* phi_host, int32_t dtype);

/* Async.  Sets u = v = u*(phi) per cell from the current phi map. */
int rdc_reset_rest(rdc_sim* sim);

/*
 * Sets the step index (steps_done of rdc_view): the index of the current
 * state, from which RDC_STOCH_ROUND derives its random stream.  To resume a
 * stochastically rounded run from a checkpoint bit for bit, restore the
 * state with rdc_set_state and the index saved with it (rdc_get_view's
 * steps_done) here.  Round-to-nearest modes do not depend on it.
 * RDC_EINVAL: sim NULL or n < 0.
 */
int rdc_set_step_index(rdc_sim* sim, int64_t n);

/*
 * Async.  Catalytic stimulation (§2): u := value (rounded to the storage
 * type) for every cell (i, j) with (i - cy)^2 + (j - cx)^2 <= r^2, the
 * squares and the sum taken in FP64 round-to-nearest with no contraction;
 * v is unchanged.  cx is the column coordinate, cy the row coordinate, cell
 * centres at integers.  Requires finite cx, cy, value and 0 <= r < 2^24;
 * cells outside the grid are skipped.
 */
int rdc_seed(rdc_sim* sim, double cx, double cy, double r, double value);

/* Async w.r.t. the device, but the host buffers are consumed before
 * return.  Sets the current state from packed H*W host arrays of dtype
 * (rounded RN-even to the storage type); u or v may be NULL to leave that
 * plane unchanged. */
int rdc_set_state(rdc_sim* sim, const void* u_host, const void* v_host,
                  int32_t dtype);

/*
 * Async.  Advances the state by n >= 0 explicit Euler steps.  Per cell, with
 * c, w, e, n_, s the current u at the cell and its west, east, north and
 * south neighbours (mirrored at the borders) and v, phi the cell's values:
 *     lap = (((w + e) + (n_ + s)) - 4 c) * (1 / (dx*dx))
 *     rat = (c - q) / (c + q)
 *     R   = (c - c*c) - (f*v + phi) * rat
 *     u'  = c + dt * (R/eps + Du*lap)     (flags drop one of the two terms)
 *     v'  = v + dt * (c - v)
 * RDC_F64 evaluates exactly this sequence in FP64 with IEEE division and no
 * fused multiply-add.  The FP32 modes evaluate, in FP32 with round-to-nearest
 * and with a = dt Du / dx^2 and b = dt / eps each computed in FP64 and rounded
 * once to FP32 (Eq. 1 scales the bracket by 1/eps):
 *     rat = (c - q) / (c + q)    (the correctly rounded quotient, as IEEE
 *                                 division gives it: see rdc_check_division)
 *     R   = fma(-fma(f, v, phi), rat, fma(-c, c, c))
 *     u'  = fma(R, b, fma(fma(-4, c, (w + e) + (n_ + s)), a, c))
 *     v'  = fma(dt, c - v, v)
 * (the flags drop the first or the second fma of u'; the kernels form R and
 * c - v with their signs flipped, which changes at most the sign of an exact
 * zero); u', v' are rounded to the storage type after every step.  Every
 * k_block and launch shape gives the same bits.
 */
int rdc_step(rdc_sim* sim, int64_t n);

/*
 * Synchronous.  Copies the current state into packed H*W host arrays of
 * dtype (RDC_DTYPE_*; values are converted from the storage type, RN-even
 * where narrowing); u_out or v_out may be NULL to skip.  Also runs the
 * health check of rdc_check and returns RDC_ENONFINITE when it fails (the
 * buffers are still filled).
 */
int rdc_read(rdc_sim* sim, void* u_out, void* v_out, int32_t dtype);

/*
 * Synchronous.  Health check: returns RDC_ENONFINITE if any cell's u is
 * non-finite or has u + q <= 0 (the pole of (u - q)/(u + q) in Eq. 1),
 * evaluated in the compute precision; *first_bad (optional) receives the
 * smallest flat index i*W + j of such a cell, or -1.
 */
int rdc_check(rdc_sim* sim, int64_t* first_bad);

/* Synchronous.  Reads u at n cells given as flat indices i*W + j into out
 * (as double).  Any index outside [0, W*H) gives RDC_EINVAL. */
int rdc_probe(rdc_sim* sim, int32_t n, const int64_t* cells, double* out);

/*
 * Halo rows of a row-strip split of one grid.  In Eq. 1 only the Laplacian
 * of u couples a row to its neighbours (v has no diffusion term and phi is
 * static), so a grid can be cut into strips of rows, each a simulation of
 * its own that holds its rows plus h halo rows copied from each neighbour:
 * stepping a strip n <= h times leaves its own rows exactly as the whole
 * grid would have them (the cut edge, a mirror border, corrupts one halo row
 * per step), and the neighbours then exchange h rows of u and v again.  The
 * paper runs one device and has no such split; these two calls are the
 * copies of that exchange.  Bitwise equality with the unsplit grid needs the
 * rows' own operation sequence, which every storage type has except under
 * RDC_STOCH_ROUND (its random words are keyed by the row index in the
 * strip).
 *
 * Async (enqueued on the simulation's stream; with pageable host memory the
 * runtime may complete the copy before returning).
 * rdc_get_rows copies rows [row0, row0 + nrows) of the current u and v into
 * u_dst and v_dst; rdc_put_rows writes them from u_src and v_src.
 *   u_*, v_* : device, pinned or pageable host memory (any pointer the
 *              runtime's unified addressing resolves), in the simulation's
 *              storage type (rdc_view.elem_bytes per value); either may be
 *              NULL to skip that plane.
 *   pitch_bytes : row stride of those buffers; 0 = packed (W * elem_bytes).
 *              A destination simulation's plane (rdc_view u/v plus
 *              row * pitch_bytes) is a valid buffer: it is current until
 *              that simulation's next rdc_step, so both simulations must
 *              share a stream (or the caller orders the two streams).
 * RDC_EINVAL: sim NULL; row0 < 0; nrows < 0; row0 + nrows > H; a nonzero
 * pitch_bytes below W * elem_bytes.  nrows = 0 does nothing.
 */
int rdc_get_rows(rdc_sim* sim, int32_t row0, int32_t nrows, void* u_dst, void* v_dst,
                 size_t pitch_bytes);
int rdc_put_rows(rdc_sim* sim, int32_t row0, int32_t nrows, const void* u_src,
                 const void* v_src, size_t pitch_bytes);

/* ---- drawing substrate (§3) ---------------------------------------------- */
/* Line width presets of §3, in cells (one pixel of the paper's simulation is
 * one cell): permeable lines slow waves, semi-permeable lines pass waves that
 * meet them head-on but not those running along them, impermeable lines stop
 * all waves. */
#define RDC_WIDTH_PERMEABLE 2
#define RDC_WIDTH_SEMIPERMEABLE 3
#define RDC_WIDTH_IMPERMEABLE 8
#define RDC_SNAP_DEGREES 15.0  /* the "snap line" angle step of §3 */

/*
 * Rotates the segment (x0,y0)-(x1,y1) about (x0,y0) to the nearest multiple of
 * snap_deg degrees, keeping its length, by exactly this FP64 sequence
 * (no contraction; C math library cos/sin/atan2/hypot/round):
 *   dx = x1 - x0; dy = y1 - y0; len = hypot(dx, dy);
 *   a = atan2(dy, dx) * (180 / pi); a = round(a / snap_deg) * snap_deg;
 *   r = a * (pi / 180); x1' = x0 + len cos(r); y1' = y0 + len sin(r).
 * Host only; no GPU needed.
 */
int rdc_snap_segment(double x0, double y0, double x1, double y1, double snap_deg,
                     double* x1_out, double* y1_out);

/*
 * Async.  Draws a straight line of substrate (§3): phi := value for every cell
 * whose centre (j, i) lies within width/2 of the segment (x0,y0)-(x1,y1)
 * (x along columns), the distance taken in FP64 without contraction:
 *   t = clamp(((j - x0) ex + (i - y0) ey) / (ex^2 + ey^2), 0, 1),
 *   (px, py) = (x0 + t ex, y0 + t ey), in if (j - px)^2 + (i - py)^2 <= (width/2)^2.
 * snap_deg > 0 first snaps the segment with rdc_snap_segment.  u and v are
 * unchanged; value must admit a rest state (as for phi maps).
 */
int rdc_draw_line(rdc_sim* sim, double x0, double y0, double x1, double y1, double width,
                  double value, double snap_deg);

/* Async.  phi := value everywhere (the filled / empty background presets of
 * §3); u and v are unchanged. */
int rdc_fill_phi(rdc_sim* sim, double value);

/* Synchronous.  Copies the phi map into a packed H*W host array of dtype
 * RDC_DTYPE_F32 or RDC_DTYPE_F64 (for saving circuits and backgrounds). */
int rdc_read_phi(rdc_sim* sim, void* out, int32_t dtype);

/* ---- outputs (§3.1) ------------------------------------------------------- */
#define RDC_RENDER_SNAPSHOT 0   /* the current state */
#define RDC_RENDER_TIMELAPSE 1  /* the timelapse record over the substrate */

/*
 * Renders a W*H RGBA8 image (row-major, 4 bytes per pixel, alpha 255) with the
 * paper's colour mapping (§3.1): red = u, green = inhibitive substrate, blue
 * = v.  Per cell, in FP32: R = rint(255 * clamp(u * u_scale, 0, 1)) (round
 * half to even), B likewise from v and v_scale, G = 255 where phi >=
 * phi_threshold (compared in FP64) else 0.  RDC_RENDER_TIMELAPSE takes R from
 * the timelapse record instead of u and sets B = 0.
 *   rgba          : host buffer (out_on_device = 0; the call synchronises) or
 *                   device buffer (out_on_device = 1, 4-byte aligned; async).
 * RDC_EINVAL for a timelapse render before any rdc_timelapse_record.
 */
int rdc_render(rdc_sim* sim, int32_t what, float u_scale, float v_scale,
               double phi_threshold, void* rgba, int32_t out_on_device);

/*
 * Async.  Timelapse (§3.1: u recorded over time, overlaid on the static
 * substrate): keeps, per cell, the running maximum of u (as FP32) over the
 * states at which this is called; reset = 1 (or the first call) restarts it
 * from the current u.  The record is allocated on first use.
 */
int rdc_timelapse_record(rdc_sim* sim, int32_t reset);

/* Waits until all work enqueued on the simulation's stream is done. */
int rdc_sync(rdc_sim* sim);

/*
 * Rest state used by the initial condition: the positive root of
 *     p(u) = u^3 + (f + q - 1) u^2 + (phi - q - f q) u - phi q,
 * which is Eq. 1's reaction bracket with v = u, times (u + q).  Found by
 * bisection on [0, 1] with a2 = (f + q) - 1, a1 = (phi - q) - f*q,
 * a0 = -(phi*q), p(x) = ((x + a2)*x + a1)*x + a0 in FP64 without
 * contraction, midpoint lo + (hi - lo)*0.5, lo := mid if p(mid) < 0 else
 * hi := mid, until the midpoint equals an end; the result is hi.  The device
 * initialiser uses the same rule, bit for bit.  RDC_EINVAL unless
 * 0 < q < 1, f + q > 1 and phi > q (1 + f).
 */
int rdc_rest_state(double phi, double f, double q, double* u_star);

/*
 * Linear stability of forward Euler at the rest state of the largest phi
 * in the map: *rho receives max |1 + dt lambda| over the eigenvalues lambda
 * of the reaction Jacobian shifted by the discrete Laplacian's spectrum
 * (from 0 to -8 Du / dx^2).  Returns RDC_EUNSTABLE_WARN when rho > 1 (the
 * homogeneous state then oscillates with period 2 instead of resting), else
 * RDC_OK.  (Table 1's phi_active gives rho < 1; phi = 0.2 gives rho > 1.)
 * The largest phi is that of the map as set, filled or read at creation; a
 * drawn line raises it when its value is larger (so after drawing it is an
 * upper bound).  The same result is recorded in rdc_view at every change of
 * phi.
 */
int rdc_stability(rdc_sim* sim, double* rho);

/* Device-side view of the current state, for zero-copy access (e.g. from
 * torch).  Pointers stay valid until the next rdc_step / rdc_destroy; the
 * current buffer alternates between the two ping-pong planes. */
typedef struct {
    void* u;              /* current u plane */
    void* v;              /* current v plane */
    const void* phi;      /* phi plane (float, or double for RDC_F64) */
    size_t pitch_bytes;   /* row stride of the state planes */
    size_t phi_pitch_bytes;
    int32_t width, height;
    int32_t precision;
    int32_t elem_bytes;   /* bytes per stored u or v value */
    int64_t steps_done;   /* step index: Euler steps applied since create / reset
                             (or as set by rdc_set_step_index) */
    int64_t launches;     /* step-kernel launches enqueued so far */
    void* stream;         /* the simulation's cudaStream_t */
    int32_t unstable;     /* 1 when forward Euler is linearly unstable at the
                             rest state of the map's largest phi (the result
                             rdc_stability returns as RDC_EUNSTABLE_WARN), or
                             when a caller-owned map has no rest state */
    int32_t reserved;
    double stability_rho; /* max |1 + dt lambda| of rdc_stability (NaN when
                             the map has no rest state) */
} rdc_view;

/* Fills *out (see rdc_view).  RDC_EINVAL if sim or out is NULL. */
int rdc_get_view(rdc_sim* sim, rdc_view* out);

/* Launch shapes of the step kernels.  They change speed only: results are
 * bitwise identical for every valid shape (each cell always runs the same
 * operation sequence on the same inputs). */
typedef struct {
    int32_t bx;        /* single-step kernel: threads per CTA along x, a
                          multiple of 32 in [32, 256]; each thread owns one
                          16-byte vector of cells (4 FP32, 2 FP64, 8 BF16/FP16) */
    int32_t rows;      /* single-step kernel: rows marched per CTA, >= 1 */
    int32_t tx, ty;    /* temporally blocked kernel: interior tile, >= 1 each */
    int32_t nthreads;  /* temporally blocked kernel: threads per CTA, a
                          multiple of 32 in [32, 512] */
    int32_t k;         /* Euler steps per launch, 1..8 (1 = single-step
                          kernel only); the tile's shared memory,
                          4 (tx + 2k)(ty + 2k) values, must fit in 227 KB */
    int32_t variant;   /* kernel for k > 1: 0 = register-streamed (every
                          intermediate level in registers; full model only,
                          test modes fall back to 1), 1 = shared-memory tile */
    int32_t krows;     /* register-streamed kernel: rows marched per CTA, >= 1 */
} rdc_launch_shape;

/*
 * Autotuner: times reps launches of each candidate shape (single step with
 * 4..32 rows per CTA; k in {2, ..., 8} with the register-streamed kernel
 * at 32..256 rows per CTA -- full model only -- and with the shared-memory
 * tile kernel; on grids so tall that a shape would need more than 65535 CTA
 * rows, that shape is skipped), keeps the fastest in cell-updates per second
 * and reports it in *out and *best_gcups (both optional).  Every timed launch
 * reads the current state and writes the spare buffers, so tuning neither
 * advances nor changes the state, and any pick gives the same bits.
 */
int rdc_tune(rdc_sim* sim, int32_t reps, rdc_launch_shape* out, double* best_gcups);

/* Current launch shapes (set at create from the grid size and k_block). */
int rdc_get_shape(rdc_sim* sim, rdc_launch_shape* out);

/* Replaces the launch shapes; RDC_EINVAL (and no change) if out of range:
 * bx not in 32..256 or not a multiple of 32, rows < 1, k outside 1..8,
 * nthreads not in 32..512 or not a multiple of 32, variant outside 0..1,
 * krows < 1, a tile needing more than 227 KB of shared memory, or (k > 1)
 * more than 65535 CTA rows at krows or ty rows each. */
int rdc_set_shape(rdc_sim* sim, const rdc_launch_shape* in);

/*
 * Allocation-free stepping (the paper has no counterpart; this is a
 * deployment convenience).  Advances caller-owned device buffers by n >= 0
 * Euler steps, exactly as rdc_step would (same kernels, same bits), and
 * allocates no device memory: no cudaMalloc, no cudaFree, no allocating
 * library call.  For callers that cannot allocate: applications whose device
 * memory is handed out by their own pool (a framework's caching allocator
 * that has reserved the device), where a library's allocation could fail or
 * fragment that pool; latency-bound loops, where cudaMalloc and cudaFree
 * would synchronise the device and stall every other stream's work; and
 * processes that must know their device footprint up front.
 *   g, p           : as rdc_create (p->k_block selects temporal blocking;
 *                    RDC_STOCH_ROUND is refused: no step index is kept);
 *   u_in, v_in     : current state, storage type of p->precision, never
 *                    written;
 *   phi            : phi map (float; double for RDC_F64) with the same pitch
 *                    in elements as the state planes;
 *   u_out, v_out   : receive the state after n steps; neither may share a
 *                    byte with any other buffer of the call (each state plane
 *                    taken as pitch_bytes * H bytes, phi as the same rows of
 *                    its elements), else RDC_EINVAL;
 *   pitch_bytes    : row stride of the state planes, a multiple of 16 and of
 *                    the element size, >= W * element size; all pointers
 *                    16-byte aligned;
 *   stream         : cudaStream_t, NULL = the legacy default stream;
 *   first_bad      : NULL to skip the health check (the call is then fully
 *                    asynchronous); otherwise the call runs the check of
 *                    rdc_check on u_out, synchronises the stream, stores the
 *                    first bad flat index (or -1) and returns
 *                    RDC_ENONFINITE if one exists.
 * Scratch: the call makes n / k + n % k launches (n with k_block <= 1).  With
 * two or more, the intermediate states live in one file-scope device array
 * of 32 MiB that every GPU loading this library holds until the process
 * exits; such a call needs 256 + 2 * roundup256(pitch_bytes * H) bytes of it
 * (FP32: just under 4 M cells, e.g. 2048 x 2047; 2048 x 2048 is 256 bytes
 * over) and larger grids get RDC_EUNSUPPORTED before anything is enqueued.
 * Calls of at most one launch use no scratch plane and take grids of any
 * size; the health check uses 8 bytes of the array.  The first call on each
 * device that uses the array looks its address up (cudaGetSymbolAddress,
 * with that device current); make that first call before any stream
 * capture.  Every call shares the array and it keeps the previous call's
 * contents (the flag is reset on every call): calls whose work overlaps on
 * the GPU -- on different streams or different threads -- race on it and
 * must be serialised by the caller.
 */
int rdc_step_noalloc(rdc_grid g, const rdc_params* p, const void* u_in,
                     const void* v_in, const void* phi, void* u_out, void* v_out,
                     size_t pitch_bytes, int64_t n, void* stream,
                     int64_t* first_bad);

/* ---- batches of independent grids ---------------------------------------- */
/*
 * A batch holds many independent simulations (parameter sweeps, interactive
 * sessions) and advances any subset of them with persistent launches over
 * all their cells at once.  Each grid has its own size, phi map and model
 * parameters (eps, f, q, Du, dt, dx); all grids of a batch share the
 * precision, the full model (flags 0) and k_block.  A grid's result is
 * bit-identical to an rdc_sim with the same parameters and inputs, whatever
 * else runs in the batch and whatever the launch configuration.
 */
typedef struct rdc_batch rdc_batch;

typedef struct {
    int32_t ngrids;        /* live grids */
    int32_t slots;         /* live + free slots; grid indices are < slots */
    int32_t precision;
    int32_t k;             /* Euler steps per launch (1 = single-step kernel) */
    int32_t rows;          /* rows per work item, single-step kernel */
    int32_t krows;         /* rows per work item, k-step kernel */
    int32_t graphs;        /* 1 = step sequences run as cached CUDA graphs */
    int32_t reserved;
    double total_cells;    /* cells over live grids */
    int64_t launches;      /* step-kernel launches enqueued so far */
    int64_t graph_launches;
    double cells_stepped;  /* cell-updates enqueued so far */
    double tuned_gcups;    /* set by rdc_batch_tune: best rate measured */
    void* stream;          /* the batch's cudaStream_t */
} rdc_batch_info;

/*
 * Creates a batch of n >= 0 grids.  grids[i], params[i] describe grid i
 * (validated as in rdc_create; params[i].precision and k_block must equal
 * params[0]'s and flags must be 0); phi_host is NULL (every map uniform
 * phi_active) or n pointers, each NULL or an H*W float map (copied).  With
 * n = 0, params must still point at one rdc_params giving the precision and
 * k_block of the grids to come.  Every grid starts at its rest state.
 * stream as for rdc_create.  Grid indices are 0..n-1.
 */
int rdc_batch_create(int32_t n, const rdc_grid* grids, const rdc_params* params,
                     const float* const* phi_host, void* stream, rdc_batch** out);

/* Adds one grid (allocates its planes; rest state) and returns its index in
 * *idx (a freed slot is reused).  The host map is validated and copied before
 * the call returns; nothing waits for the device: the planes come from the
 * batch's stream-ordered memory pool and their initialisation (phi upload,
 * rest state) is enqueued on the batch's stream behind the work already there
 * (from page-locked host memory the map's copy is asynchronous too).
 * RDC_ENOMEM if the device memory is short. */
int rdc_batch_add(rdc_batch* b, rdc_grid g, const rdc_params* p, const float* phi_host,
                  int32_t* idx);

/* Removes grid idx; its memory returns to the batch's pool once the work
 * enqueued on the batch's stream before this call has finished (the call does
 * not wait), and the slot can take a new grid at once. */
int rdc_batch_remove(rdc_batch* b, int32_t idx);

/* Waits for the batch's stream, frees everything.  NULL is a no-op. */
void rdc_batch_destroy(rdc_batch* b);

/* Async.  Stimulation of grid idx, as rdc_seed. */
int rdc_batch_seed(rdc_batch* b, int32_t idx, double cx, double cy, double r, double value);

/* Sets grid idx's step index, as rdc_set_step_index (for resuming a
 * stochastically rounded grid from a checkpoint). */
int rdc_batch_set_step_index(rdc_batch* b, int32_t idx, int64_t n);

/* Sets grid idx's current state from packed host arrays, as rdc_set_state. */
int rdc_batch_set_state(rdc_batch* b, int32_t idx, const void* u_host, const void* v_host,
                        int32_t dtype);

/*
 * Async.  Advances the m grids idx[0..m-1] (distinct, live; idx = NULL: every
 * live grid) by n >= 0 Euler steps: n / k launches of the k-step kernel and
 * n % k single-step launches, each a persistent launch over the warp-sized
 * tiles of exactly those grids (the call's tile map, uploaded on the batch's
 * stream).  With graphs on (the default) the launch sequence for a given
 * (n, shape) is captured once into a CUDA graph and replayed for any subset;
 * adding or removing a grid discards the graphs.
 */
int rdc_batch_step(rdc_batch* b, const int32_t* idx, int32_t m, int64_t n);

/* Synchronous.  Health check of grid idx, as rdc_check. */
int rdc_batch_check(rdc_batch* b, int32_t idx, int64_t* first_bad);

/* Synchronous.  Grid idx's state into host arrays, as rdc_read. */
int rdc_batch_read(rdc_batch* b, int32_t idx, void* u_out, void* v_out, int32_t dtype);

/* Waits for the batch's stream. */
int rdc_batch_sync(rdc_batch* b);

/* Launch configuration: k (1..8), rows and krows (>= 1), graphs (0/1).  Any
 * valid configuration gives the same bits. */
int rdc_batch_set_config(rdc_batch* b, int32_t k, int32_t rows, int32_t krows, int32_t graphs);

/* Fills *out with the batch's configuration and counters (rdc_batch_info).
 * RDC_EINVAL if b or out is NULL. */
int rdc_batch_get_info(rdc_batch* b, rdc_batch_info* out);

/* Host only.  Width and height of grid idx (the sizes of the host arrays that
 * rdc_batch_set_state and rdc_batch_read take).  RDC_EINVAL if b or out is
 * NULL or idx is not a live grid. */
int rdc_batch_get_grid(rdc_batch* b, int32_t idx, rdc_grid* out);

/* Stability of forward Euler at the rest state of grid idx's largest phi,
 * as rdc_stability (recorded when the grid was added): *rho receives max
 * |1 + dt lambda|; returns RDC_EUNSTABLE_WARN when rho > 1, else RDC_OK;
 * RDC_EINVAL if b or rho is NULL or idx is not a live grid. */
int rdc_batch_stability(rdc_batch* b, int32_t idx, double* rho);

/*
 * Autotuner: times reps launches of each candidate (single step with 8, 16 or
 * 32 rows per item; k in {2, 3, 4, 5, 6, 8} with 32..256 rows per item) over all
 * live grids, keeps the fastest in cell-updates per second, and reports it in
 * *out (optional).  Every timed launch reads the current buffers and writes
 * the spare ones, so tuning does not advance or change any grid's state.
 */
int rdc_batch_tune(rdc_batch* b, int32_t reps, rdc_batch_info* out);

/* ---- diagnostics --------------------------------------------------------- */
/*
 * The paper has no counterpart: a self-check of this library's arithmetic.
 * The FP32 modes compute the ratio (c - q)/(c + q) of rdc_step with a refined
 * hardware reciprocal and one Markstein correction of the quotient (P.
 * Markstein, IBM J. Res. Dev. 34(1), 1990) instead of the compiler's division
 * sequence.  That yields the IEEE-754 round-to-nearest quotient whenever the
 * refined reciprocal is itself correctly rounded.  This call checks, on the
 * current device and bit for bit against the CUDA runtime's IEEE intrinsics:
 *   [0] the refined reciprocal of every b = 2^e (1 + m 2^-23) with e in
 *       [-125, 125] (every significand; b and 1/b normal);
 *   [1] the ratio, in the scalar and the paired form the kernels use, for
 *       every FP32 c with 0 < c + q < 2^126, q rounded to FP32 as the kernels
 *       round it (about 2.1e9 values for q = 0.002; beyond 2^126 the
 *       reciprocal estimate flushes the subnormal 1/(c + q) to zero, where
 *       c*c has long overflowed and the state is non-finite anyway);
 *   [2] a / b for n_random pairs of random normal floats (exponents in
 *       [-60, 60], random signs; a SplitMix64 stream from seed); 0 skips it.
 * out->checked[i] and out->mismatches[i] count the values of part i;
 * out->first_bad[i] is the smallest offending bit pattern of b [0] or c [1],
 * or the smallest offending pair index [2]; 0xffffffff when there is none.
 * Synchronous (tens of milliseconds); allocates and frees a few bytes of
 * device memory.  RDC_EINVAL: out NULL, or q not a finite value > 0.
 */
typedef struct {
    uint64_t checked[3];
    uint64_t mismatches[3];
    uint32_t first_bad[3];
    uint32_t reserved;
} rdc_division_report;

int rdc_check_division(double q, uint64_t n_random, uint64_t seed, rdc_division_report* out);

/*
 * The paper has no counterpart: exposes the stochastic rounding of
 * RDC_STOCH_ROUND.  For i in 0..n-1, rounds the FP32 value x[i] to the
 * storage type of `precision` (RDC_F32_BF16STORE or RDC_F32_F16STORE) as the
 * step kernels round the new u (u_out[i]) and the new v (v_out[i]) of the
 * cell in column col0 + i, row `row`, when they write the state with index
 * `step` under key `seed`; the results are widened back to float.  Host
 * arrays of n floats (copied).  Synchronous; allocates and frees device
 * memory.  RDC_EINVAL: another precision, n < 0, col0 or row < 0, col0 + n
 * beyond 2^31 - 1, or a NULL array with n > 0.
 */
int rdc_stoch_round_sample(int32_t precision, uint32_t seed, int64_t step, int32_t row,
                           int32_t col0, int32_t n, const float* x, float* u_out,
                           float* v_out);

/*
 * The paper has no counterpart: exposes the Philox4x32-10 generator (Salmon
 * et al., SC'11) whose words drive RDC_STOCH_ROUND, so that it can be checked
 * against the generator's published known-answer vectors.  For i in 0..n-1,
 * out[4i .. 4i+3] receives the four output words for counter ctr[4i .. 4i+3]
 * and key key[2i], key[2i+1], computed on the current device by the function
 * the step kernels call.  Host arrays (copied).  Synchronous; allocates and
 * frees device memory.  RDC_EINVAL: n < 0, n > 2^24, or a NULL array with
 * n > 0.
 */
int rdc_philox_sample(int32_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/* Human-readable name of a status code (static storage). */
const char* rdc_status_str(int status);

/* Message of the last CUDA failure seen on this thread (static storage, ""
 * if none). */
const char* rdc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RDC_H_ */
