// Host-side interface between the C ABI (rdc_api.cu) and the kernel
// translation units.  Not installed; not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace rdc {

// Model constants in FP64 as given by the caller; each launcher rounds them
// to its compute precision.
struct ModelD {
    double eps, f, q, Du, dt, inv_dx2;
    int sr = 0;           // 1: stochastic rounding to the 16-bit storage type
    unsigned seed = 0;    // key of the rounding stream
    long long step0 = 0;  // index of the state a launch reads; level l writes step0 + l
    int flip = 0;         // single-step kernel: row blocks in reverse order
};

// Which terms of u_t a step evaluates (match the RDC_*_ONLY flags), plus
// MODE_SR for stochastic rounding to the storage type.
enum { MODE_FULL = 0, MODE_DIFFUSION = 1, MODE_REACTION = 2, MODE_SR = 4 };

// Storage codes (match RDC_F32 ... RDC_F32_F16STORE).
enum Prec { P_F32 = 0, P_F64 = 1, P_BF16 = 2, P_F16 = 3 };

// Launch shape of the single-step kernel: bx threads per CTA along x (a
// multiple of 32, each thread owning one 16-byte vector of cells), each CTA
// marching `rows` rows.
struct Shape1 {
    int bx;
    int rows;
};

// Temporal blocking, k Euler steps per launch (1..8).  variant 0: the
// register-streamed kernel (full model only), each CTA marching `krows` rows;
// variant 1: the shared-memory tile kernel with tx x ty interior cells and
// nthreads threads (a multiple of 32).
struct ShapeK {
    int tx, ty, k, nthreads;
    int variant = 0;
    int krows = 256;
};

// Geometry of one grid's planes.  All planes share the row pitch `pitch`
// counted in elements of their own type.
struct Planes {
    const void* u;
    const void* v;
    const void* phi;
    void* u1;
    void* v1;
    int W, H;
    int64_t pitch;
};

// One grid of a batch, as the batched kernels read it from device memory.
// par is the index (0/1) of the current buffer when the batch launch
// sequence starts; launch j of a sequence reads buffer (par + j) & 1 and
// writes the other.  The grids a call steps are those of its tile map, so
// one captured graph serves any subset.  Model constants stay FP64 here and
// are rounded to the compute precision per work item, exactly as the
// single-grid launchers do.
struct GridDesc {
    void* u[2];
    void* v[2];
    const void* phi;
    int W, H;
    long long pitch;  // elements, all planes
    double eps, f, q, Du, dt, inv_dx2;
    int par;
    int active;       // 1: stepped by the current call (host bookkeeping; the
                      // kernels take the call's grids from its tile map)
    unsigned seed;    // stochastic rounding key (RDC_STOCH_ROUND)
    int pad_;
    long long steps;  // Euler steps taken by the grid before the current call
};

// The work of a batched launch: every grid of the call cut into tiles of
// `cols` x `rows` cells (the last column and row of tiles partial), one tile
// per work item of a warp:
//   single step : cols = 32 * VEC cells (one 16-byte vector per lane)
//   streamed k  : cols = OUTC output columns
// The tiles of the call's grids are numbered consecutively, grid after grid,
// row-major within a grid; span i lists grid g_i, its tiles per row, and the
// number of the grid's first tile.  The map holds only the grids the call
// steps, so a launch over a few grids of a large batch touches nothing else.
struct TileSpan {
    int g;        // grid (slot) index into the descriptor table
    int tiles_x;  // tiles per row of that grid
    int first;    // number of its first tile
    int pad;
};
struct TileMap {
    int nspans;   // grids in the call
    int total;    // tiles in the call (the work items)
    int pad[2];
    TileSpan span[1];  // nspans entries (the map is allocated for its capacity)
};

// Kernels of rdc_step_*.cu.
cudaError_t launch_step1(int prec, int mode, const Planes& g, const ModelD& m,
                         Shape1 s, cudaStream_t st);
cudaError_t launch_stepk(int prec, int mode, const Planes& g, const ModelD& m,
                         ShapeK s, cudaStream_t st);
size_t stepk_smem_bytes(int prec, ShapeK s);
cudaError_t launch_stream(int prec, const Planes& g, const ModelD& m, int k, int rows,
                          cudaStream_t st);
// Batched launches over the tiles of a device tile map, `rows` rows per tile
// (persistent: `ctas` CTAs of 128 threads; each warp takes the next tile from
// the work queue `queue`, two zeroed counters that the launch leaves zeroed);
// launch index j selects buffers.  sbase: Euler steps of the call before this launch (the rounding
// stream's step index is the grid's steps + sbase + level); sr: stochastic
// rounding.
cudaError_t launch_batch_step1(int prec, const GridDesc* d, const TileMap* map, int rows,
                               unsigned* queue, int j, long long sbase, int sr, int ctas,
                               cudaStream_t st);
cudaError_t launch_batch_stream(int prec, const GridDesc* d, const TileMap* map, int rows,
                                unsigned* queue, int k, int j, long long sbase, int sr,
                                int ctas, cudaStream_t st);
// Columns a warp covers (single step) / writes (streamed, k steps).
int batch_step1_cols(int prec);
int batch_stream_outc(int prec, int k, bool sr);
// The kernel that rdc_step uses for one launch of k > 1 steps.
cudaError_t launch_kblock(int prec, int mode, const Planes& g, const ModelD& m,
                          ShapeK s, cudaStream_t st);

// Kernels of rdc_aux.cu.
cudaError_t launch_rest(int prec, void* u, void* v, const void* phi, int W,
                        int H, int64_t pitch, double f, double q,
                        cudaStream_t st);
cudaError_t launch_seed(int prec, void* u, int W, int H, int64_t pitch,
                        double cx, double cy, double r, double value,
                        cudaStream_t st);
// Health: atomically lowers *first_bad to the smallest flat index whose u is
// non-finite or has u + q <= 0 (caller initialises it to ~0ull).
cudaError_t launch_health(int prec, const void* u, int W, int H, int64_t pitch,
                          double q, unsigned long long* first_bad,
                          cudaStream_t st);
// *out := max(*out, the bit pattern of the largest phi of the map as a
// double, ordered as a signed integer; see k_phi_max).  The caller
// initialises *out to LLONG_MIN.
cudaError_t launch_phi_max(int prec, const void* phi, int W, int H, int64_t pitch,
                           long long* out, cudaStream_t st);
// Packed host-order buffer of dtype `src_dtype` -> pitched plane of storage
// `prec` (RN-even); and back.
cudaError_t launch_pack_in(int prec, int src_dtype, const void* src, void* dst,
                           int W, int H, int64_t pitch, cudaStream_t st);
cudaError_t launch_pack_out(int prec, int dst_dtype, const void* src, void* dst,
                            int W, int H, int64_t pitch, cudaStream_t st);
// phi: packed float/double host-order -> pitched phi plane of `prec`.
cudaError_t launch_phi_in(int prec, int src_dtype, const void* src, void* dst,
                          int W, int H, int64_t pitch, cudaStream_t st);
// phi plane := value (uniform map).
cudaError_t launch_fill_phi(int prec, void* dst, int W, int H, int64_t pitch, double value,
                            cudaStream_t st);
// phi := value for cells within width/2 of the segment (x0,y0)-(x1,y1).
cudaError_t launch_draw_line(int prec, void* phi, int W, int H, int64_t pitch, double x0,
                             double y0, double x1, double y1, double width, double value,
                             cudaStream_t st);
// RGBA8 image of the state (or of the timelapse plane tl when non-null).
cudaError_t launch_render(int prec, const void* u, const void* v, const void* phi,
                          const float* tl, int W, int H, int64_t pitch, int64_t tl_pitch,
                          float u_scale, float v_scale, double thr, void* out, cudaStream_t st);
// tl := reset ? u : max(tl, u), in FP32.
cudaError_t launch_timelapse(int prec, const void* u, float* tl, int W, int H, int64_t pitch,
                             int64_t tl_pitch, int reset, cudaStream_t st);
// u at flat cell indices -> doubles.
cudaError_t launch_probe(int prec, const void* u, int W, int64_t pitch,
                         const int64_t* cells, int n, double* out,
                         cudaStream_t st);

// Element sizes.
inline int state_bytes(int prec) { return prec == P_F64 ? 8 : (prec == P_F32 ? 4 : 2); }
inline int phi_bytes(int prec) { return prec == P_F64 ? 8 : 4; }
inline int vec_cells(int prec) { return 16 / state_bytes(prec); }
inline int dtype_bytes(int dtype) { return dtype == 1 ? 8 : (dtype == 0 ? 4 : 2); }

}  // namespace rdc
