// Auxiliary kernels of librdc: rest-state initialisation, catalytic
// stimulation (§2), the health flag, dtype conversion between packed host
// order and the pitched device planes, and probe gathers.
#include <climits>
#include <cmath>

#include "rdc_device.cuh"
#include "rdc_internal.h"

namespace rdc {

// ---------------------------------------------------------------------------
// conversions by host dtype code (RDC_DTYPE_F32/F64/BF16/F16)
// ---------------------------------------------------------------------------

template <typename D>
__device__ __forceinline__ D cvt_from_double(double x);
template <>
__device__ __forceinline__ float cvt_from_double<float>(double x) { return __double2float_rn(x); }
template <>
__device__ __forceinline__ double cvt_from_double<double>(double x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_from_double<__nv_bfloat16>(double x) { return __double2bfloat16(x); }
template <>
__device__ __forceinline__ __half cvt_from_double<__half>(double x) { return __double2half(x); }

__device__ __forceinline__ double to_double(float x) { return (double)x; }
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
__device__ __forceinline__ double to_double(__half x) { return (double)__half2float(x); }

// Direct single-rounding conversion Src -> Dst (every narrower value is
// exactly representable in double, so going through double rounds once).
template <typename Dst, typename Src>
__device__ __forceinline__ Dst convert(Src x)
{
    return cvt_from_double<Dst>(to_double(x));
}

// ---------------------------------------------------------------------------
// rest state
// ---------------------------------------------------------------------------

// Positive root of p(u) = u^3 + (f+q-1) u^2 + (phi-q-fq) u - phi q (Eq. 1's
// reaction bracket with v = u, times u + q) by the bisection rule documented
// at rdc_rest_state: FP64, one rounding per operation, no contraction.
__device__ __forceinline__ double rest_root(double phi, double f, double q)
{
    const double a2 = __dsub_rn(__dadd_rn(f, q), 1.0);
    const double a1 = __dsub_rn(__dsub_rn(phi, q), __dmul_rn(f, q));
    const double a0 = -__dmul_rn(phi, q);
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 2000; ++it) {
        const double mid = __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), 0.5));
        if (mid == lo || mid == hi) break;
        const double p = __dadd_rn(
            __dmul_rn(__dadd_rn(__dmul_rn(__dadd_rn(mid, a2), mid), a1), mid), a0);
        if (p < 0.0) lo = mid; else hi = mid;
    }
    return hi;
}

template <typename S>
__global__ void k_rest(S* __restrict__ u, S* __restrict__ v,
                       const typename Traits<S>::PhiT* __restrict__ phi, int W,
                       int H, int64_t pitch, double f, double q)
{
    // Each thread keeps the last phi it met and that phi's root; a warp runs
    // the bisection only when one of its lanes meets a new value (phi maps
    // are piecewise constant, so most warps skip it).  The loop keeps whole
    // warps together so the vote covers every lane.
    const int64_t n = (int64_t)W * H;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double last_phi = NAN, last_root = 0.0;
    for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); k0 < n;
         k0 += stride) {
        const int64_t k = k0 + (threadIdx.x & 31);
        const bool live = k < n;
        int64_t o = 0;
        double ph = last_phi;
        if (live) {
            const int64_t i = k / W, j = k - i * W;
            o = i * pitch + j;
            ph = (double)phi[o];
        }
        const bool need = live && !(ph == last_phi);
        if (__any_sync(0xffffffffu, need) && need) {
            last_root = rest_root(ph, f, q);
            last_phi = ph;
        }
        if (live) {
            const S s = cvt_from_double<S>(last_root);
            u[o] = s;
            v[o] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// stimulation (§2): u := value inside a disk
// ---------------------------------------------------------------------------

template <typename S>
__global__ void k_seed(S* __restrict__ u, int W, int H, int64_t pitch,
                       int i0, int j0, int ni, int nj, double cx, double cy,
                       double r2, S value)
{
    const int64_t n = (int64_t)ni * nj;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int i = i0 + (int)(k / nj);
        const int j = j0 + (int)(k % nj);
        const double dy = __dsub_rn((double)i, cy);
        const double dx = __dsub_rn((double)j, cx);
        if (__dadd_rn(__dmul_rn(dy, dy), __dmul_rn(dx, dx)) <= r2)
            u[(int64_t)i * pitch + j] = value;
    }
}

// ---------------------------------------------------------------------------
// health flag
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool bad_cell(float x, float q) { return !isfinite(x) || !(__fadd_rn(x, q) > 0.0f); }
__device__ __forceinline__ bool bad_cell(double x, double q) { return !isfinite(x) || !(__dadd_rn(x, q) > 0.0); }

template <typename S>
__global__ void k_health(const S* __restrict__ u, int W, int H, int64_t pitch,
                         typename Traits<S>::T q, unsigned long long* first_bad)
{
    const int64_t n = (int64_t)W * H;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / W, j = k - i * W;
        if (bad_cell(widen(u[i * pitch + j]), q))
            atomicMin(first_bad, (unsigned long long)k);
    }
}

// Largest phi of a pitched map, as the bit pattern of a double: for IEEE
// doubles of equal sign the bit patterns, read as signed 64-bit integers,
// order like the values, and every negative value orders below every positive
// one, so an atomic maximum over the patterns is the maximum value (a NaN with
// the sign bit clear orders above +infinity and is reported as such).
template <typename P>
__global__ void k_phi_max(const P* __restrict__ phi, int W, int H, int64_t pitch,
                          long long* out)
{
    const int64_t n = (int64_t)W * H;
    long long m = LLONG_MIN;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / W, j = k - i * W;
        const double x = (double)phi[i * pitch + j];
        const long long b = __double_as_longlong(x);
        // negative values: flip the magnitude bits so that they order too
        m = max(m, b >= 0 ? b : (long long)(b ^ 0x7FFFFFFFFFFFFFFFLL));
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ---------------------------------------------------------------------------
// packed <-> pitched conversion
// ---------------------------------------------------------------------------

template <typename Src, typename Dst>
__global__ void k_pack_in(const Src* __restrict__ src, Dst* __restrict__ dst,
                          int W, int H, int64_t pitch)
{
    const int64_t n = (int64_t)W * H;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / W, j = k - i * W;
        dst[i * pitch + j] = convert<Dst>(src[k]);
    }
}

template <typename Src, typename Dst>
__global__ void k_pack_out(const Src* __restrict__ src, Dst* __restrict__ dst,
                           int W, int H, int64_t pitch)
{
    const int64_t n = (int64_t)W * H;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / W, j = k - i * W;
        dst[k] = convert<Dst>(src[i * pitch + j]);
    }
}

template <typename S>
__global__ void k_probe(const S* __restrict__ u, int W, int64_t pitch,
                        const int64_t* __restrict__ cells, int n,
                        double* __restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        const int64_t c = cells[k];
        const int64_t i = c / W, j = c - i * W;
        out[k] = to_double(u[i * pitch + j]);
    }
}

// ---------------------------------------------------------------------------
// drawing substrate (§3): phi := value within width/2 of a segment
// ---------------------------------------------------------------------------

template <typename P>
__global__ void k_draw_line(P* __restrict__ phi, int W, int H, int64_t pitch, int i0, int j0,
                            int ni, int nj, double x0, double y0, double x1, double y1,
                            double half2, P value)
{
    const double ex = __dsub_rn(x1, x0), ey = __dsub_rn(y1, y0);
    const double L2 = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
    const int64_t n = (int64_t)ni * nj;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int i = i0 + (int)(k / nj);
        const int j = j0 + (int)(k % nj);
        const double x = (double)j, y = (double)i;
        double t = 0.0;
        if (L2 > 0.0)
            t = __ddiv_rn(__dadd_rn(__dmul_rn(__dsub_rn(x, x0), ex), __dmul_rn(__dsub_rn(y, y0), ey)),
                          L2);
        t = fmin(fmax(t, 0.0), 1.0);
        const double px = __dadd_rn(x0, __dmul_rn(t, ex));
        const double py = __dadd_rn(y0, __dmul_rn(t, ey));
        const double dx = __dsub_rn(x, px), dy = __dsub_rn(y, py);
        if (__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= half2)
            phi[(int64_t)i * pitch + j] = value;
    }
}

// ---------------------------------------------------------------------------
// rendering (§3.1): red = u, green = inhibitive substrate, blue = v
// ---------------------------------------------------------------------------

// 255 * clamp(x * scale, 0, 1) rounded half to even, all in FP32.
__device__ __forceinline__ unsigned int chan(float x, float scale)
{
    const float y = fminf(fmaxf(__fmul_rn(x, scale), 0.0f), 1.0f);
    return (unsigned int)__float2int_rn(__fmul_rn(255.0f, y));
}

// Four consecutive pixels of row i starting at column j0 (a multiple of 4):
// u, v (or the timelapse record) and phi in vectors where the four lie inside
// the grid, one 16-byte store when the output allows it.  HBM-bound: reads
// the state and phi once, writes 4 bytes per pixel.
// Four values from p (n of them inside the grid), widened to float; one
// 16-byte (FP32) or 8-byte (16-bit) load when all four are inside.  Row
// starts are 16-byte aligned for FP32 and 8-byte aligned for 16-bit storage
// (the row pitch is a multiple of 16 bytes) and j0 is a multiple of 4.
template <typename S>
__device__ __forceinline__ void load4(const S* p, int n, float (&x)[4])
{
    if (n == 4) {
        if constexpr (sizeof(S) == 4) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(p));
            x[0] = q.x;
            x[1] = q.y;
            x[2] = q.z;
            x[3] = q.w;
            return;
        } else if constexpr (sizeof(S) == 2) {
            union {
                uint2 d;
                S h[4];
            } q;
            q.d = __ldg(reinterpret_cast<const uint2*>(p));
#pragma unroll
            for (int e = 0; e < 4; ++e) x[e] = (float)widen(q.h[e]);
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) x[e] = e < n ? (float)widen(p[e]) : 0.0f;
}

// The green channel: phi >= thr compared in FP64.  For a float phi the
// launcher passes thr_f, the smallest float >= thr, and phi >= thr_f in FP32
// is the same test (GB300's FP64 pipe would otherwise bound the kernel).
template <typename P>
__device__ __forceinline__ void green4(const P* p, int n, double thr, float thr_f,
                                       unsigned int (&g)[4])
{
    if constexpr (sizeof(P) == 4) {
        float f[4];
        load4(p, n, f);
#pragma unroll
        for (int e = 0; e < 4; ++e) g[e] = (f[e] >= thr_f) ? 255u : 0u;
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) g[e] = (e < n && p[e] >= thr) ? 255u : 0u;
    }
}

template <typename S>
__global__ void k_render(const S* __restrict__ u, const S* __restrict__ v,
                         const typename Traits<S>::PhiT* __restrict__ phi,
                         const float* __restrict__ tl, int W, int H, int64_t pitch,
                         int64_t tl_pitch, float u_scale, float v_scale, double thr,
                         float thr_f, uchar4* __restrict__ out, int vec_out)
{
    const int j0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (j0 >= W) return;
    const int n = min(4, W - j0);
    for (int i = blockIdx.y; i < H; i += gridDim.y) {
        const int64_t o = (int64_t)i * pitch + j0;
        float a[4], b[4];
        unsigned int g[4];
        if (tl) {  // timelapse: running maximum of u over the static substrate
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                a[e] = e < n ? tl[(int64_t)i * tl_pitch + j0 + e] : 0.0f;
                b[e] = 0.0f;
            }
        } else {
            load4(u + o, n, a);
            load4(v + o, n, b);
        }
        green4(phi + o, n, thr, thr_f, g);
        unsigned int px[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const unsigned int r = chan(a[e], u_scale);
            const unsigned int bl = tl ? 0u : chan(b[e], v_scale);
            px[e] = r | (g[e] << 8) | (bl << 16) | (255u << 24);
        }
        uchar4* dst = out + (int64_t)i * W + j0;
        if (vec_out && n == 4) {
            *reinterpret_cast<uint4*>(dst) = make_uint4(px[0], px[1], px[2], px[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (e < n) *reinterpret_cast<unsigned int*>(dst + e) = px[e];
        }
    }
}

template <typename S>
__global__ void k_timelapse(const S* __restrict__ u, float* __restrict__ tl, int W, int H,
                            int64_t pitch, int64_t tl_pitch, int reset)
{
    const int j0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (j0 >= W) return;
    const int n = min(4, W - j0);
    for (int i = blockIdx.y; i < H; i += gridDim.y) {
        float x[4];
        load4(u + (int64_t)i * pitch + j0, n, x);
        float* t = tl + (int64_t)i * tl_pitch + j0;
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (e < n) t[e] = reset ? x[e] : fmaxf(t[e], x[e]);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;  // grid-stride beyond 32 CTAs per SM
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_rest(int prec, void* u, void* v, const void* phi, int W,
                        int H, int64_t pitch, double f, double q,
                        cudaStream_t st)
{
    const int t = 256;
    const int b = grid_for((int64_t)W * H, t);
    switch (prec) {
        case P_F32: k_rest<float><<<b, t, 0, st>>>((float*)u, (float*)v, (const float*)phi, W, H, pitch, f, q); break;
        case P_F64: k_rest<double><<<b, t, 0, st>>>((double*)u, (double*)v, (const double*)phi, W, H, pitch, f, q); break;
        case P_BF16: k_rest<__nv_bfloat16><<<b, t, 0, st>>>((__nv_bfloat16*)u, (__nv_bfloat16*)v, (const float*)phi, W, H, pitch, f, q); break;
        case P_F16: k_rest<__half><<<b, t, 0, st>>>((__half*)u, (__half*)v, (const float*)phi, W, H, pitch, f, q); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_seed(int prec, void* u, int W, int H, int64_t pitch,
                        double cx, double cy, double r, double value,
                        cudaStream_t st)
{
    // bounding box of the disk, clipped to the grid (all in FP64; the box is
    // one cell wider than needed on each side, the kernel decides membership)
    double lo_i = floor(cy - r) - 1.0, hi_i = ceil(cy + r) + 1.0;
    double lo_j = floor(cx - r) - 1.0, hi_j = ceil(cx + r) + 1.0;
    if (lo_i < 0.0) lo_i = 0.0;
    if (lo_j < 0.0) lo_j = 0.0;
    if (hi_i > H - 1) hi_i = H - 1;
    if (hi_j > W - 1) hi_j = W - 1;
    if (hi_i < lo_i || hi_j < lo_j) return cudaSuccess;  // disk misses the grid
    const int i0 = (int)lo_i, j0 = (int)lo_j;
    const int ni = (int)hi_i - i0 + 1, nj = (int)hi_j - j0 + 1;
    const double r2 = r * r;
    const int t = 256;
    const int b = grid_for((int64_t)ni * nj, t);
    switch (prec) {
        case P_F32: k_seed<float><<<b, t, 0, st>>>((float*)u, W, H, pitch, i0, j0, ni, nj, cx, cy, r2, (float)value); break;
        case P_F64: k_seed<double><<<b, t, 0, st>>>((double*)u, W, H, pitch, i0, j0, ni, nj, cx, cy, r2, value); break;
        case P_BF16: k_seed<__nv_bfloat16><<<b, t, 0, st>>>((__nv_bfloat16*)u, W, H, pitch, i0, j0, ni, nj, cx, cy, r2, __double2bfloat16(value)); break;
        case P_F16: k_seed<__half><<<b, t, 0, st>>>((__half*)u, W, H, pitch, i0, j0, ni, nj, cx, cy, r2, __double2half(value)); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_health(int prec, const void* u, int W, int H, int64_t pitch,
                          double q, unsigned long long* first_bad,
                          cudaStream_t st)
{
    const int t = 256;
    const int b = grid_for((int64_t)W * H, t);
    switch (prec) {
        case P_F32: k_health<float><<<b, t, 0, st>>>((const float*)u, W, H, pitch, (float)q, first_bad); break;
        case P_F64: k_health<double><<<b, t, 0, st>>>((const double*)u, W, H, pitch, q, first_bad); break;
        case P_BF16: k_health<__nv_bfloat16><<<b, t, 0, st>>>((const __nv_bfloat16*)u, W, H, pitch, (float)q, first_bad); break;
        case P_F16: k_health<__half><<<b, t, 0, st>>>((const __half*)u, W, H, pitch, (float)q, first_bad); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_phi_max(int prec, const void* phi, int W, int H, int64_t pitch,
                           long long* out, cudaStream_t st)
{
    const int t = 256;
    const int b = grid_for((int64_t)W * H, t);
    if (prec == P_F64)
        k_phi_max<double><<<b, t, 0, st>>>((const double*)phi, W, H, pitch, out);
    else
        k_phi_max<float><<<b, t, 0, st>>>((const float*)phi, W, H, pitch, out);
    return cudaGetLastError();
}

template <typename Src>
static cudaError_t pack_in_src(int prec, const void* src, void* dst, int W, int H,
                               int64_t pitch, int b, int t, cudaStream_t st)
{
    const Src* s = (const Src*)src;
    switch (prec) {
        case P_F32: k_pack_in<Src, float><<<b, t, 0, st>>>(s, (float*)dst, W, H, pitch); break;
        case P_F64: k_pack_in<Src, double><<<b, t, 0, st>>>(s, (double*)dst, W, H, pitch); break;
        case P_BF16: k_pack_in<Src, __nv_bfloat16><<<b, t, 0, st>>>(s, (__nv_bfloat16*)dst, W, H, pitch); break;
        case P_F16: k_pack_in<Src, __half><<<b, t, 0, st>>>(s, (__half*)dst, W, H, pitch); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_in(int prec, int src_dtype, const void* src, void* dst,
                           int W, int H, int64_t pitch, cudaStream_t st)
{
    const int t = 256;
    const int b = grid_for((int64_t)W * H, t);
    switch (src_dtype) {
        case 0: return pack_in_src<float>(prec, src, dst, W, H, pitch, b, t, st);
        case 1: return pack_in_src<double>(prec, src, dst, W, H, pitch, b, t, st);
        case 2: return pack_in_src<__nv_bfloat16>(prec, src, dst, W, H, pitch, b, t, st);
        case 3: return pack_in_src<__half>(prec, src, dst, W, H, pitch, b, t, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename S>
static cudaError_t pack_out_src(int dst_dtype, const void* src, void* dst, int W,
                                int H, int64_t pitch, int b, int t, cudaStream_t st)
{
    const S* s = (const S*)src;
    switch (dst_dtype) {
        case 0: k_pack_out<S, float><<<b, t, 0, st>>>(s, (float*)dst, W, H, pitch); break;
        case 1: k_pack_out<S, double><<<b, t, 0, st>>>(s, (double*)dst, W, H, pitch); break;
        case 2: k_pack_out<S, __nv_bfloat16><<<b, t, 0, st>>>(s, (__nv_bfloat16*)dst, W, H, pitch); break;
        case 3: k_pack_out<S, __half><<<b, t, 0, st>>>(s, (__half*)dst, W, H, pitch); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_out(int prec, int dst_dtype, const void* src, void* dst,
                            int W, int H, int64_t pitch, cudaStream_t st)
{
    const int t = 256;
    const int b = grid_for((int64_t)W * H, t);
    switch (prec) {
        case P_F32: return pack_out_src<float>(dst_dtype, src, dst, W, H, pitch, b, t, st);
        case P_F64: return pack_out_src<double>(dst_dtype, src, dst, W, H, pitch, b, t, st);
        case P_BF16: return pack_out_src<__nv_bfloat16>(dst_dtype, src, dst, W, H, pitch, b, t, st);
        case P_F16: return pack_out_src<__half>(dst_dtype, src, dst, W, H, pitch, b, t, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_phi_in(int prec, int src_dtype, const void* src, void* dst,
                          int W, int H, int64_t pitch, cudaStream_t st)
{
    const int t = 256;
    const int b = grid_for((int64_t)W * H, t);
    const bool dbl = (prec == P_F64);
    if (src_dtype == 0) {
        if (dbl) k_pack_in<float, double><<<b, t, 0, st>>>((const float*)src, (double*)dst, W, H, pitch);
        else k_pack_in<float, float><<<b, t, 0, st>>>((const float*)src, (float*)dst, W, H, pitch);
    } else if (src_dtype == 1) {
        if (dbl) k_pack_in<double, double><<<b, t, 0, st>>>((const double*)src, (double*)dst, W, H, pitch);
        else k_pack_in<double, float><<<b, t, 0, st>>>((const double*)src, (float*)dst, W, H, pitch);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename P>
__global__ void k_fill(P* __restrict__ dst, int W, int H, int64_t pitch, P value)
{
    const int64_t n = (int64_t)W * H;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / W, j = k - i * W;
        dst[i * pitch + j] = value;
    }
}

cudaError_t launch_fill_phi(int prec, void* dst, int W, int H, int64_t pitch,
                            double value, cudaStream_t st)
{
    const int t = 256;
    const int b = grid_for((int64_t)W * H, t);
    if (prec == P_F64)
        k_fill<double><<<b, t, 0, st>>>((double*)dst, W, H, pitch, value);
    else
        k_fill<float><<<b, t, 0, st>>>((float*)dst, W, H, pitch, (float)value);
    return cudaGetLastError();
}

cudaError_t launch_draw_line(int prec, void* phi, int W, int H, int64_t pitch, double x0,
                             double y0, double x1, double y1, double width, double value,
                             cudaStream_t st)
{
    const double h = 0.5 * width;
    double lo_i = floor(fmin(y0, y1) - h) - 1.0, hi_i = ceil(fmax(y0, y1) + h) + 1.0;
    double lo_j = floor(fmin(x0, x1) - h) - 1.0, hi_j = ceil(fmax(x0, x1) + h) + 1.0;
    if (lo_i < 0.0) lo_i = 0.0;
    if (lo_j < 0.0) lo_j = 0.0;
    if (hi_i > H - 1) hi_i = H - 1;
    if (hi_j > W - 1) hi_j = W - 1;
    if (hi_i < lo_i || hi_j < lo_j) return cudaSuccess;  // misses the grid
    const int i0 = (int)lo_i, j0 = (int)lo_j;
    const int ni = (int)hi_i - i0 + 1, nj = (int)hi_j - j0 + 1;
    const int t = 256;
    const int b = grid_for((int64_t)ni * nj, t);
    const double half2 = h * h;
    if (prec == P_F64)
        k_draw_line<double><<<b, t, 0, st>>>((double*)phi, W, H, pitch, i0, j0, ni, nj, x0, y0, x1, y1, half2, value);
    else
        k_draw_line<float><<<b, t, 0, st>>>((float*)phi, W, H, pitch, i0, j0, ni, nj, x0, y0, x1, y1, half2, (float)value);
    return cudaGetLastError();
}

cudaError_t launch_render(int prec, const void* u, const void* v, const void* phi,
                          const float* tl, int W, int H, int64_t pitch, int64_t tl_pitch,
                          float u_scale, float v_scale, double thr, void* out, cudaStream_t st)
{
    const int t = 128;
    const dim3 grid((unsigned)(((W + 3) / 4 + t - 1) / t), (unsigned)min(H, 65535));
    uchar4* o = (uchar4*)out;
    const int vec = ((uintptr_t)out % 16 == 0) && (W % 4 == 0);
    // smallest float >= thr (for float phi maps)
    float thr_f = (float)thr;
    if ((double)thr_f < thr) thr_f = std::nextafter(thr_f, INFINITY);
    switch (prec) {
        case P_F32: k_render<float><<<grid, t, 0, st>>>((const float*)u, (const float*)v, (const float*)phi, tl, W, H, pitch, tl_pitch, u_scale, v_scale, thr, thr_f, o, vec); break;
        case P_F64: k_render<double><<<grid, t, 0, st>>>((const double*)u, (const double*)v, (const double*)phi, tl, W, H, pitch, tl_pitch, u_scale, v_scale, thr, thr_f, o, vec); break;
        case P_BF16: k_render<__nv_bfloat16><<<grid, t, 0, st>>>((const __nv_bfloat16*)u, (const __nv_bfloat16*)v, (const float*)phi, tl, W, H, pitch, tl_pitch, u_scale, v_scale, thr, thr_f, o, vec); break;
        case P_F16: k_render<__half><<<grid, t, 0, st>>>((const __half*)u, (const __half*)v, (const float*)phi, tl, W, H, pitch, tl_pitch, u_scale, v_scale, thr, thr_f, o, vec); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_timelapse(int prec, const void* u, float* tl, int W, int H, int64_t pitch,
                             int64_t tl_pitch, int reset, cudaStream_t st)
{
    const int t = 128;
    const dim3 grid((unsigned)(((W + 3) / 4 + t - 1) / t), (unsigned)min(H, 65535));
    switch (prec) {
        case P_F32: k_timelapse<float><<<grid, t, 0, st>>>((const float*)u, tl, W, H, pitch, tl_pitch, reset); break;
        case P_F64: k_timelapse<double><<<grid, t, 0, st>>>((const double*)u, tl, W, H, pitch, tl_pitch, reset); break;
        case P_BF16: k_timelapse<__nv_bfloat16><<<grid, t, 0, st>>>((const __nv_bfloat16*)u, tl, W, H, pitch, tl_pitch, reset); break;
        case P_F16: k_timelapse<__half><<<grid, t, 0, st>>>((const __half*)u, tl, W, H, pitch, tl_pitch, reset); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_probe(int prec, const void* u, int W, int64_t pitch,
                         const int64_t* cells, int n, double* out,
                         cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int t = 128;
    const int b = (n + t - 1) / t;
    switch (prec) {
        case P_F32: k_probe<float><<<b, t, 0, st>>>((const float*)u, W, pitch, cells, n, out); break;
        case P_F64: k_probe<double><<<b, t, 0, st>>>((const double*)u, W, pitch, cells, n, out); break;
        case P_BF16: k_probe<__nv_bfloat16><<<b, t, 0, st>>>((const __nv_bfloat16*)u, W, pitch, cells, n, out); break;
        case P_F16: k_probe<__half><<<b, t, 0, st>>>((const __half*)u, W, pitch, cells, n, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rdc
