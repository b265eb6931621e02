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
};

// Storage codes (match RDC_F32 ... RDC_F32_F16STORE).
enum Prec { P_F32 = 0, P_F64 = 1, P_BF16 = 2, P_F16 = 3 };

// Launch shape of the single-step kernel: bx threads per CTA along x (a
// multiple of 32, each thread owning one 16-byte vector of cells), each CTA
// marching `rows` rows.
struct Shape1 {
    int bx;
    int rows;
};

// Tile of the temporally blocked kernel: tx x ty interior cells per CTA,
// k Euler steps per launch (1..8), nthreads threads (a multiple of 32).
struct ShapeK {
    int tx, ty, k, nthreads;
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

// Kernels of rdc_step_*.cu.
cudaError_t launch_step1(int prec, int mode, const Planes& g, const ModelD& m,
                         Shape1 s, cudaStream_t st);
cudaError_t launch_stepk(int prec, int mode, const Planes& g, const ModelD& m,
                         ShapeK s, cudaStream_t st);
size_t stepk_smem_bytes(int prec, ShapeK s);

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
// Packed host-order buffer of dtype `src_dtype` -> pitched plane of storage
// `prec` (RN-even); and back.
cudaError_t launch_pack_in(int prec, int src_dtype, const void* src, void* dst,
                           int W, int H, int64_t pitch, cudaStream_t st);
cudaError_t launch_pack_out(int prec, int dst_dtype, const void* src, void* dst,
                            int W, int H, int64_t pitch, cudaStream_t st);
// phi: packed float/double host-order -> pitched phi plane of `prec`.
cudaError_t launch_phi_in(int prec, int src_dtype, const void* src, void* dst,
                          int W, int H, int64_t pitch, cudaStream_t st);
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
