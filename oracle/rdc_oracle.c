/*
 * FP64 CPU oracle for the two-variable Oregonator reaction-diffusion step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * constant or helper with the CUDA library, and it includes nothing from it.
 *
 * Build:  gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC rdc_oracle.c -lm
 * (-ffp-contract=off matters: aarch64 GCC contracts a*b+c into an FMA by
 * default, which would change the rounding of every expression below.)
 *
 * The model (Eq. 1, §2):
 *     u_t = (1/eps) [ u - u^2 - (f v + phi) (u - q)/(u + q) ] + Du lap(u)
 *     v_t = u - v
 * integrated with explicit forward Euler, timestep dt, and the five-node
 * discrete Laplace operator on a grid of spacing dx (§2, paragraph after
 * Table 1).  Default values are Table 1.  Catalytic stimulation sets u of the
 * stimulated cells to a value (§2 uses 1.0).
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes of the repository):
 *   - borders: zero flux, implemented as a cell-centred mirror ghost (the
 *     out-of-range neighbour takes the value of the border cell itself);
 *   - update order: Jacobi -- u' and v' are both computed from step n;
 *   - summation order of the Laplacian: ((w + e) + (n + s)) - 4 c, then times
 *     1/(dx*dx) computed once; this order makes a uniform field's Laplacian
 *     exactly zero and keeps the result invariant under the 8 symmetries of
 *     the square;
 *   - the reaction bracket is evaluated as (c - c*c) - (f*v + phi) * rat with
 *     rat = (c - q)/(c + q), then divided by eps;
 *   - initial state: the homogeneous rest state u = v = u*(phi), u* the
 *     positive root of the reaction term with v = u (see orc_rest_state);
 *   - no clamping of u or v.
 *
 * Grid layout: row-major, cell (i, j) = row i (y), column j (x), flat index
 * i*W + j, no padding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Model parameters.  Field order is part of the ctypes binding in
 * oracle/__init__.py. */
typedef struct {
    double eps;  /* time-scale ratio epsilon (Table 1: 0.0243) */
    double f;    /* stoichiometric factor (Table 1: 1.4) */
    double q;    /* propagation scaling factor (Table 1: 0.002) */
    double Du;   /* diffusion coefficient of u (Table 1: 0.45) */
    double dt;   /* Euler timestep (Table 1: 0.001) */
    double dx;   /* grid spacing (Table 1: 0.25) */
    int32_t flags; /* ORC_DIFFUSION_ONLY / ORC_REACTION_ONLY test modes */
    int32_t pad_;
} orc_params;

enum { ORC_DIFFUSION_ONLY = 1, ORC_REACTION_ONLY = 2 };

/* Status codes. */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENONFINITE = 4 };

/* ------------------------------------------------------------------------- */
/* Rest state (initial condition reading, Eq. 1 with u_t = v_t = 0)          */
/* ------------------------------------------------------------------------- */

/*
 * Homogeneous rest state of Eq. 1: with no spatial variation and v_t = 0 we
 * need v = u, and u_t = 0 needs the reaction bracket to vanish:
 *     u - u^2 - (f u + phi)(u - q)/(u + q) = 0.
 * Multiplying by (u + q) > 0 gives the cubic
 *     p(u) = u^3 + (f + q - 1) u^2 + (phi - q - f q) u - phi q = 0,
 * which has exactly one positive root when f + q > 1 and phi > q (1 + f)
 * (one sign change in its coefficients).  p(0) = -phi q < 0 and
 * p(1) = (f + phi)(1 - q) > 0 for 0 < q < 1, so the root lies in (0, 1).
 *
 * The root is found by bisection on [0, 1] with the polynomial evaluated by
 * Horner's rule in this exact order:
 *     a2 = (f + q) - 1;  a1 = (phi - q) - f*q;  a0 = -(phi*q);
 *     p(x) = ((x + a2)*x + a1)*x + a0
 * and midpoints mid = lo + (hi - lo)*0.5; if p(mid) < 0 then lo = mid else
 * hi = mid; the loop stops when mid equals lo or hi, and the result is hi.
 * The result is therefore a fully specified double, the same on every IEEE
 * machine, which any other implementation of this rule must reproduce bit
 * for bit.
 */
int orc_rest_state(double phi, double f, double q, double* u_star)
{
    if (!u_star) return ORC_EINVAL;
    if (!(q > 0.0 && q < 1.0) || !((f + q) > 1.0) || !(phi > q * (1.0 + f)))
        return ORC_EINVAL;
    const double a2 = (f + q) - 1.0;
    const double a1 = (phi - q) - f * q;
    const double a0 = -(phi * q);
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 2000; ++it) {
        double mid = lo + (hi - lo) * 0.5;
        if (mid == lo || mid == hi) break;
        double p = ((mid + a2) * mid + a1) * mid + a0;
        if (p < 0.0) lo = mid; else hi = mid;
    }
    *u_star = hi;
    return ORC_OK;
}

/* Fills u = v = u*(phi[k]) for every cell. */
int orc_rest_field(int64_t n, const double* phi, double f, double q,
                   double* u, double* v)
{
    if (n < 0 || (n > 0 && (!phi || !u || !v))) return ORC_EINVAL;
    for (int64_t k = 0; k < n; ++k) {
        double s;
        int rc = orc_rest_state(phi[k], f, q, &s);
        if (rc) return rc;
        u[k] = s;
        v[k] = s;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Stimulation (§2: the excitatory concentration u of stimulated cells is    */
/* set to a value)                                                           */
/* ------------------------------------------------------------------------- */

/*
 * Sets u := value for every cell (i, j) with (i - cy)^2 + (j - cx)^2 <= r^2,
 * cell centres at integer coordinates, cx along columns (x), cy along rows
 * (y).  v is left untouched.  Returns the number of cells set.
 */
int64_t orc_seed_disk(int32_t W, int32_t H, double* u, double cx, double cy,
                      double r, double value)
{
    if (W < 1 || H < 1 || !u || !(r >= 0.0)) return -1;
    int64_t count = 0;
    const double r2 = r * r;
    for (int32_t i = 0; i < H; ++i) {
        for (int32_t j = 0; j < W; ++j) {
            double dy = (double)i - cy;
            double dx = (double)j - cx;
            if (dy * dy + dx * dx <= r2) {
                u[(int64_t)i * W + j] = value;
                ++count;
            }
        }
    }
    return count;
}

/* ------------------------------------------------------------------------- */
/* One explicit Euler step (§2) of Eq. 1                                     */
/* ------------------------------------------------------------------------- */

static int params_ok(const orc_params* p)
{
    if (!p) return 0;
    const double vals[6] = {p->eps, p->f, p->q, p->Du, p->dt, p->dx};
    for (int k = 0; k < 6; ++k)
        if (!isfinite(vals[k])) return 0;
    if (!(p->eps > 0.0) || !(p->q > 0.0) || !(p->dt > 0.0) || !(p->dx > 0.0))
        return 0;
    if (p->Du < 0.0) return 0;
    return 1;
}

/* The state is healthy while u is finite and stays right of the pole of
 * (u - q)/(u + q) at u = -q (Eq. 1). */
static int cell_bad(double u, double q)
{
    return !isfinite(u) || (u + q) <= 0.0;
}

/* One row of the step.  Returns the first column whose new u is unhealthy,
 * or -1. */
static int32_t step_row(int32_t W, int32_t H, int32_t i, const orc_params* p,
                        double inv_dx2, const double* phi, const double* u,
                        const double* v, double* u1, double* v1)
{
    const double eps = p->eps, f = p->f, q = p->q, Du = p->Du, dt = p->dt;
    const int use_react = !(p->flags & ORC_DIFFUSION_ONLY);
    const int use_diff = !(p->flags & ORC_REACTION_ONLY);
    const int32_t in = (i > 0) ? i - 1 : 0;          /* mirror ghost */
    const int32_t is = (i < H - 1) ? i + 1 : H - 1;  /* mirror ghost */
    int32_t first_bad = -1;
    for (int32_t j = 0; j < W; ++j) {
        const int32_t jw = (j > 0) ? j - 1 : 0;
        const int32_t je = (j < W - 1) ? j + 1 : W - 1;
        const int64_t k = (int64_t)i * W + j;
        const double c = u[k];
        const double w = u[(int64_t)i * W + jw];
        const double e = u[(int64_t)i * W + je];
        const double nn = u[(int64_t)in * W + j];
        const double s = u[(int64_t)is * W + j];
        const double vc = v[k];

        /* five-node Laplacian, zero-flux borders */
        const double lap = (((w + e) + (nn + s)) - 4.0 * c) * inv_dx2;
        /* reaction bracket of Eq. 1 */
        const double rat = (c - q) / (c + q);
        const double R = (c - c * c) - (f * vc + phi[k]) * rat;

        double du;
        if (use_react && use_diff)
            du = R / eps + Du * lap;
        else if (use_react)
            du = R / eps;
        else if (use_diff)
            du = Du * lap;
        else
            du = 0.0;
        const double un = c + dt * du;
        u1[k] = un;
        v1[k] = vc + dt * (c - vc);
        if (first_bad < 0 && cell_bad(un, q)) first_bad = j;
    }
    return first_bad;
}

/*
 * One step from (u, v) to (u1, v1); the output arrays must not alias the
 * input ones.  *bad_index receives the flat index of the first cell (in
 * row-major order) whose new u is non-finite or has u + q <= 0, else -1.
 * nthreads <= 1 runs single-threaded; rows are independent (Jacobi), so the
 * result does not depend on nthreads.
 */
int orc_step(int32_t W, int32_t H, const orc_params* p, const double* phi,
             const double* u, const double* v, double* u1, double* v1,
             int32_t nthreads, int64_t* bad_index)
{
    if (W < 1 || H < 1 || !params_ok(p) || !phi || !u || !v || !u1 || !v1)
        return ORC_EINVAL;
    const double inv_dx2 = 1.0 / (p->dx * p->dx);
    int64_t first_bad = -1;
#ifdef _OPENMP
    if (nthreads > 1) {
        int64_t best = INT64_MAX;
#pragma omp parallel for num_threads(nthreads) schedule(static) reduction(min : best)
        for (int32_t i = 0; i < H; ++i) {
            int32_t jb = step_row(W, H, i, p, inv_dx2, phi, u, v, u1, v1);
            if (jb >= 0) {
                int64_t kk = (int64_t)i * W + jb;
                if (kk < best) best = kk;
            }
        }
        first_bad = (best == INT64_MAX) ? -1 : best;
    } else
#endif
    {
        (void)nthreads;
        for (int32_t i = 0; i < H; ++i) {
            int32_t jb = step_row(W, H, i, p, inv_dx2, phi, u, v, u1, v1);
            if (jb >= 0 && first_bad < 0) first_bad = (int64_t)i * W + jb;
        }
    }
    if (bad_index) *bad_index = first_bad;
    return first_bad >= 0 ? ORC_ENONFINITE : ORC_OK;
}

/*
 * nsteps Euler steps in place on (u, v).  Stops after the first step that
 * leaves an unhealthy cell; *bad_step receives that step (1-based) and
 * *bad_index the cell, else both -1.
 *
 * With nprobe > 0 it also records, for each probe cell probe[m], the
 * arrival time of the first upward crossing of theta: the first step n with
 * u_n >= theta, linearly interpolated between steps n-1 and n, i.e.
 *     t = (n - 1) + (theta - u_{n-1}) / (u_n - u_{n-1})   (in steps),
 * 0 if the probe already starts at or above theta, -1 if it never crosses.
 */
int orc_run(int32_t W, int32_t H, const orc_params* p, const double* phi,
            double* u, double* v, int64_t nsteps, int32_t nthreads,
            int32_t nprobe, const int64_t* probe, double theta, double* t_arr,
            int64_t* bad_step, int64_t* bad_index)
{
    if (W < 1 || H < 1 || nsteps < 0 || !params_ok(p) || !phi || !u || !v)
        return ORC_EINVAL;
    if (nprobe < 0 || (nprobe > 0 && (!probe || !t_arr))) return ORC_EINVAL;
    const int64_t n = (int64_t)W * H;
    for (int32_t m = 0; m < nprobe; ++m)
        if (probe[m] < 0 || probe[m] >= n) return ORC_EINVAL;
    if (bad_step) *bad_step = -1;
    if (bad_index) *bad_index = -1;
    for (int32_t m = 0; m < nprobe; ++m)
        t_arr[m] = (u[probe[m]] >= theta) ? 0.0 : -1.0;

    double* u1 = (double*)malloc(sizeof(double) * (size_t)n);
    double* v1 = (double*)malloc(sizeof(double) * (size_t)n);
    if (!u1 || !v1) {
        free(u1);
        free(v1);
        return ORC_ENOMEM;
    }
    int rc = ORC_OK;
    for (int64_t step = 1; step <= nsteps; ++step) {
        int64_t bi = -1;
        int src = orc_step(W, H, p, phi, u, v, u1, v1, nthreads, &bi);
        for (int32_t m = 0; m < nprobe; ++m) {
            if (t_arr[m] >= 0.0) continue;
            const double a = u[probe[m]], b = u1[probe[m]];
            if (b >= theta)
                t_arr[m] = (double)(step - 1) + (theta - a) / (b - a);
        }
        memcpy(u, u1, sizeof(double) * (size_t)n);
        memcpy(v, v1, sizeof(double) * (size_t)n);
        if (src != ORC_OK) {
            if (bad_step) *bad_step = step;
            if (bad_index) *bad_index = bi;
            rc = src;
            break;
        }
    }
    free(u1);
    free(v1);
    return rc;
}

/* Number of threads the OpenMP runtime offers (1 without OpenMP). */
int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Outputs (§3.1): red = u, green = inhibitive substrate, blue = v           */
/* ------------------------------------------------------------------------- */

/* 255 * clamp(x * scale, 0, 1), rounded half to even; every step in FP32
 * (the paper fixes no precision for the picture; the CUDA path renders in
 * FP32, and an 8-bit code must be decided in one precision on both sides). */
static unsigned char orc_chan(float x, float scale)
{
    float y = x * scale;
    if (y < 0.0f) y = 0.0f;
    if (y > 1.0f) y = 1.0f;
    return (unsigned char)lrintf(255.0f * y);
}

/* RGBA8 image (row-major, 4 bytes per cell).  tl == NULL: R from u, B from
 * v; otherwise R from the timelapse record tl and B = 0.  G = 255 where
 * phi >= thr (in FP64), else 0.  A = 255. */
void orc_render(int64_t n, const float* u, const float* v, const double* phi,
                const float* tl, float u_scale, float v_scale, double thr,
                unsigned char* out)
{
    for (int64_t k = 0; k < n; ++k) {
        unsigned char r, b;
        if (tl) {
            r = orc_chan(tl[k], u_scale);
            b = 0;
        } else {
            r = orc_chan(u[k], u_scale);
            b = orc_chan(v[k], v_scale);
        }
        out[4 * k + 0] = r;
        out[4 * k + 1] = (phi[k] >= thr) ? 255 : 0;
        out[4 * k + 2] = b;
        out[4 * k + 3] = 255;
    }
}

/* Timelapse record: tl := u (reset) or max(tl, u), per cell, in FP32. */
void orc_timelapse(int64_t n, const float* u, float* tl, int32_t reset)
{
    for (int64_t k = 0; k < n; ++k)
        tl[k] = (reset || u[k] > tl[k]) ? u[k] : tl[k];
}

/* ------------------------------------------------------------------------- */
/* Drawing substrate (§3): lines of a given width, optional angle snapping   */
/* ------------------------------------------------------------------------- */

/* Rotates (x0,y0)-(x1,y1) about (x0,y0) to the nearest multiple of snap
 * degrees, keeping its length (the app's "snap line", 15 degrees). */
int orc_snap_segment(double x0, double y0, double x1, double y1, double snap,
                     double* x1o, double* y1o)
{
    if (!x1o || !y1o || !(snap > 0.0)) return ORC_EINVAL;
    const double dx = x1 - x0, dy = y1 - y0;
    const double len = hypot(dx, dy);
    double a = atan2(dy, dx) * (180.0 / 3.14159265358979323846);
    a = round(a / snap) * snap;
    const double r = a * (3.14159265358979323846 / 180.0);
    *x1o = x0 + len * cos(r);
    *y1o = y0 + len * sin(r);
    return ORC_OK;
}

/* phi := value for every cell whose centre (x = j, y = i) lies within
 * width/2 of the segment: the nearest point of the segment is x0 + t e with
 * t the clamped projection of the cell onto e = (x1 - x0, y1 - y0).
 * Returns the number of cells set. */
int64_t orc_draw_line(int32_t W, int32_t H, double* phi, double x0, double y0,
                      double x1, double y1, double width, double value)
{
    if (W < 1 || H < 1 || !phi || !(width >= 0.0)) return -1;
    const double ex = x1 - x0, ey = y1 - y0;
    const double L2 = ex * ex + ey * ey;
    const double h = 0.5 * width;
    const double half2 = h * h;
    int64_t count = 0;
    for (int32_t i = 0; i < H; ++i) {
        for (int32_t j = 0; j < W; ++j) {
            const double x = (double)j, y = (double)i;
            double t = 0.0;
            if (L2 > 0.0) t = ((x - x0) * ex + (y - y0) * ey) / L2;
            if (t < 0.0) t = 0.0;
            if (t > 1.0) t = 1.0;
            const double px = x0 + t * ex, py = y0 + t * ey;
            const double dx = x - px, dy = y - py;
            if (dx * dx + dy * dy <= half2) {
                phi[(int64_t)i * W + j] = value;
                ++count;
            }
        }
    }
    return count;
}

/* ------------------------------------------------------------------------
 * Stochastic rounding to 16-bit storage (the RDC_STOCH_ROUND variant of the
 * storage conversion).  The paper stores nothing in reduced precision; this
 * is the rounding rule of the variant, written from its definition:
 *   lo = x rounded toward zero onto the target grid, hi = the next grid
 *   value away from zero; result hi iff r16 < 2^16 (|x| - |lo|) / (|hi| -
 *   |lo|), else lo; non-finite x, and FP16 at or beyond 65504, round to
 *   nearest.
 * The random words are Philox4x32-10 (J. K. Salmon, M. A. Moraes, R. O.
 * Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 * ------------------------------------------------------------------------ */

/* Philox4x32 with 10 rounds.  One round: the products M0 * c0 and M1 * c2
 * (64-bit); the new counter is (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),
 * hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); then the key advances by the Weyl
 * increments.  M0 = 0xD2511F53, M1 = 0xCD9E8D57, increments 0x9E3779B9 and
 * 0xBB67AE85 (the constants of the paper's Philox4x32). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t n1 = (uint32_t)p1;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        const uint32_t n3 = (uint32_t)p0;
        c[0] = n0;
        c[1] = n1;
        c[2] = n2;
        c[3] = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    memcpy(out, c, sizeof c);
}

/* Grid spacing of the target format at |x| (x finite, nonzero or zero):
 * mant = stored significand bits, emin = smallest normal exponent. */
static double orc_spacing(double ax, int mant, int emin)
{
    int e = emin;
    if (ax >= ldexp(1.0, emin)) {
        (void)frexp(ax, &e); /* ax = m 2^e, m in [0.5, 1) */
        e -= 1;              /* ax in [2^e, 2^(e+1)) */
    }
    return ldexp(1.0, e - mant);
}

/* fmt 0: BF16 (8 significant bits, exponent range of FP32);
 * fmt 1: FP16 (11 significant bits, smallest normal 2^-14, largest 65504). */
float orc_round_stoch(float x, uint32_t r16, int32_t fmt)
{
    const int mant = fmt == 0 ? 7 : 10;
    const int emin = fmt == 0 ? -126 : -14;
    const double xd = (double)x;
    if (isnan(xd)) return x;
    const double ax = fabs(xd);
    const double sgn = signbit(xd) ? -1.0 : 1.0;
    if (fmt == 1 && !(ax < 65504.0)) {
        if (isinf(ax)) return x;
        /* RN: 65504 below the midpoint 65520, infinity from it (the tie goes
         * to the even significand, which is the next binade) */
        return (float)(sgn * (ax < 65520.0 ? 65504.0 : INFINITY));
    }
    if (isinf(ax)) return x;
    const double sp = orc_spacing(ax, mant, emin);
    const double lo = floor(ax / sp) * sp;
    if (lo == ax) return x;
    const double frac = (ax - lo) / sp; /* exact: sp is a power of two */
    double mag = ((double)r16 < ldexp(frac, 16)) ? lo + sp : lo;
    if (fmt == 0 && mag >= ldexp(1.0, 128)) mag = INFINITY;
    return (float)(sgn * mag);
}

/* The rounding of the u (out_u) and the v (out_v) of cells (col0 + i, row)
 * for the state with index `step`, key seed: counter (col / 4, row, step mod
 * 2^32, step / 2^32), key (seed, 0); word col mod 4 of the output, its top
 * 16 bits for u and its low 16 bits for v. */
void orc_round_stoch_cells(int64_t n, const float* x, uint32_t seed, int64_t step, int32_t row,
                           int32_t col0, int32_t fmt, float* out_u, float* out_v)
{
    for (int64_t i = 0; i < n; ++i) {
        const int64_t col = (int64_t)col0 + i;
        const uint64_t s = (uint64_t)step;
        const uint32_t ctr[4] = {(uint32_t)(col / 4), (uint32_t)row, (uint32_t)s,
                                 (uint32_t)(s >> 32)};
        const uint32_t key[2] = {seed, 0u};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        const uint32_t word = w[col % 4];
        out_u[i] = orc_round_stoch(x[i], word >> 16, fmt);
        out_v[i] = orc_round_stoch(x[i], word & 0xFFFFu, fmt);
    }
}
