// Diagnostics of the step kernels' arithmetic: rdc_check_division checks
// the FP32 division exhaustively, rdc_stoch_round_sample exposes the
// stochastic rounding of RDC_STOCH_ROUND and rdc_philox_sample the
// Philox4x32-10 generator behind it.
//
// rdc_check_division: exhaustive device check of the FP32 division that
// every FP32 step kernel uses for the ratio (u - q)/(u + q) of Eq. 1.
//
// The kernels divide with a refined reciprocal and one Markstein correction
// (div_rn in rdc_device.cuh) instead of the compiler's IEEE division.  That
// is the IEEE-754 round-to-nearest quotient when the refined reciprocal is
// itself correctly rounded; this file checks both steps against the CUDA
// runtime's IEEE intrinsics (__frcp_rn, __fdiv_rn), over
//   [0] every significand of b at every exponent whose reciprocal is normal
//       (the refined reciprocal rcp_rn),
//   [1] every finite FP32 u with 0 < u + q < 2^126, i.e. every operand pair
//       the cell update can form with the given q short of u ~ 1e38 (where
//       1/(u + q) is subnormal, the estimate flushes it to zero, and u*u has
//       long overflowed anyway) -- div_rn and the paired div2_rn,
//   [2] random normal operand pairs (a counter-based SplitMix64 stream).
#include <cmath>
#include <type_traits>

#include "rdc.h"
#include "rdc_device.cuh"
#include "rdc_host.h"

namespace rdc {
namespace {

constexpr int kExpLo = -125, kExpHi = 125;  // 2^e: b and 1/b both normal

struct Counts {
    unsigned long long checked[3];
    unsigned long long bad[3];
    unsigned int first_bad[3];
};

__device__ __forceinline__ void flush(Counts* out, int i, unsigned long long checked,
                                      unsigned long long bad, unsigned int first)
{
    atomicAdd(&out->checked[i], checked);
    if (bad) {
        atomicAdd(&out->bad[i], bad);
        atomicMin(&out->first_bad[i], first);
    }
}

__device__ __forceinline__ bool same(float a, float b)
{
    return __float_as_uint(a) == __float_as_uint(b);
}

// [0] b = 2^e * (1 + m / 2^23) for every m and e in [kExpLo, kExpHi].
__global__ void k_check_rcp(Counts* out)
{
    const uint64_t total = uint64_t(kExpHi - kExpLo + 1) << 23;
    unsigned long long n = 0, bad = 0;
    unsigned int first = 0xffffffffu;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned int m = (unsigned int)(i & 0x7fffffu);
        const int e = kExpLo + (int)(i >> 23);
        const float b = __uint_as_float(((unsigned int)(e + 127) << 23) | m);
        ++n;
        if (!same(rcp_rn(b), __frcp_rn(b))) {
            ++bad;
            first = min(first, __float_as_uint(b));
        }
    }
    flush(out, 0, n, bad, first);
}

// [1] every bit pattern of u, in pairs (2p, 2p + 1) so that the paired
// division is checked on the same operands.
__global__ void k_check_ratio(float q, Counts* out)
{
    unsigned long long n = 0, bad = 0;
    unsigned int first = 0xffffffffu;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < (1ull << 31);
         p += (uint64_t)gridDim.x * blockDim.x) {
        const float u0 = __uint_as_float((unsigned int)(2 * p));
        const float u1 = __uint_as_float((unsigned int)(2 * p + 1));
        const float2 a = make_float2(__fadd_rn(u0, -q), __fadd_rn(u1, -q));
        const float2 b = make_float2(__fadd_rn(u0, q), __fadd_rn(u1, q));
        const float2 nb = make_float2(__fadd_rn(-u0, -q), __fadd_rn(-u1, -q));
        const float2 r2 = div2_rn(a, b, nb);
        const float uu[2] = {u0, u1}, aa[2] = {a.x, a.y}, bb[2] = {b.x, b.y},
                    rr[2] = {r2.x, r2.y};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!isfinite(uu[h]) || !(bb[h] > 0.0f) || !(bb[h] < 0x1p126f)) continue;
            ++n;
            const float ref = __fdiv_rn(aa[h], bb[h]);
            if (!same(div_rn(aa[h], bb[h]), ref) || !same(rr[h], ref)) {
                ++bad;
                first = min(first, __float_as_uint(uu[h]));
            }
        }
    }
    flush(out, 1, n, bad, first);
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// A normal float with a random sign, exponent in [-60, 60] and significand.
__device__ __forceinline__ float random_normal(uint64_t r)
{
    const unsigned int e = 127 - 60 + (unsigned int)((r >> 23) % 121u);
    return __uint_as_float(((unsigned int)(r >> 40) & 0x80000000u) | (e << 23) |
                           (unsigned int)(r & 0x7fffffu));
}

// [2] n random pairs (a, b) from the stream seed.
__global__ void k_check_random(uint64_t n_pairs, uint64_t seed, Counts* out)
{
    unsigned long long n = 0, bad = 0;
    unsigned int first = 0xffffffffu;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_pairs;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const float a = random_normal(splitmix64(seed + 2 * i));
        const float b = random_normal(splitmix64(seed + 2 * i + 1));
        ++n;
        if (!same(div_rn(a, b), __fdiv_rn(a, b))) {
            ++bad;
            first = min(first, (unsigned int)i);
        }
    }
    flush(out, 2, n, bad, first);
}

// The rounding of the step kernels for the u and the v of cells
// (col0 + i, row) writing state `step`.
template <typename S>
__global__ void k_sr_sample(const float* __restrict__ x, int n, unsigned seed, long long step,
                            int row, int col0, float* __restrict__ uo, float* __restrict__ vo)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int col = col0 + i;
    const unsigned w = sr_word(sr_quad_bits(seed, col >> 2, row, step), col & 3);
    // the forms the step kernels take: the integer ones where they apply
    // (BF16 unless NaN, FP16 in its normal range), the general one otherwise
    const float xi = x[i];
    if (std::is_same_v<S, __nv_bfloat16> && !isnan(xi)) {
        uo[i] = sr_bf16(xi, w >> 16);
        vo[i] = sr_bf16(xi, w & 0xFFFFu);
    } else if (std::is_same_v<S, __half> && fp16_normal(xi)) {
        uo[i] = sr_f16_normal(xi, w >> 16);
        vo[i] = sr_f16_normal(xi, w & 0xFFFFu);
    } else {
        uo[i] = quantize_sr<S>(xi, w);
        vo[i] = quantize_sr<S>(xi, w << 16);
    }
}

// Philox4x32-10 outputs for n given counters and keys, computed by the very
// function the stochastically rounding step kernels call.
__global__ void k_philox_sample(const unsigned* __restrict__ ctr,
                                const unsigned* __restrict__ key, int n,
                                unsigned* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Philox4 c{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    const Philox4 r = philox4x32_10(c, key[2 * i], key[2 * i + 1]);
    out[4 * i] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

}  // namespace
}  // namespace rdc

using namespace rdc;

extern "C" int rdc_philox_sample(int32_t n, const uint32_t* ctr, const uint32_t* key,
                                 uint32_t* out)
{
    if (n < 0 || n > (1 << 24) || (n > 0 && (!ctr || !key || !out))) return RDC_EINVAL;
    if (n == 0) return RDC_OK;
    int rc = host_check_device();
    if (rc) return rc;
    unsigned* d = nullptr;
    const size_t words = (size_t)n * 10;  // 4 counter, 2 key, 4 output words each
    cudaError_t e = cudaMalloc((void**)&d, words * sizeof(unsigned));
    if (e != cudaSuccess) return host_cuda_fail(e, "cudaMalloc(philox sample)");
    unsigned* dc = d;
    unsigned* dk = d + 4 * (size_t)n;
    unsigned* dout = d + 6 * (size_t)n;
    do {
        if ((e = cudaMemcpy(dc, ctr, 4 * (size_t)n * sizeof(unsigned),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            break;
        if ((e = cudaMemcpy(dk, key, 2 * (size_t)n * sizeof(unsigned),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            break;
        const int bs = 256, gs = (n + bs - 1) / bs;
        k_philox_sample<<<gs, bs>>>(dc, dk, n, dout);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        e = cudaMemcpy(out, dout, 4 * (size_t)n * sizeof(unsigned), cudaMemcpyDeviceToHost);
    } while (false);
    cudaFree(d);
    return e == cudaSuccess ? RDC_OK : host_cuda_fail(e, "philox sample");
}

extern "C" int rdc_stoch_round_sample(int32_t precision, uint32_t seed, int64_t step,
                                      int32_t row, int32_t col0, int32_t n, const float* x,
                                      float* u_out, float* v_out)
{
    if ((precision != RDC_F32_BF16STORE && precision != RDC_F32_F16STORE) || n < 0 ||
        col0 < 0 || row < 0 || (int64_t)col0 + n > 2147483647LL ||
        (n > 0 && (!x || !u_out || !v_out)))
        return RDC_EINVAL;
    if (n == 0) return RDC_OK;
    int rc = host_check_device();
    if (rc) return rc;
    float* d = nullptr;
    const size_t bytes = (size_t)n * sizeof(float);
    cudaError_t e = cudaMalloc((void**)&d, 3 * bytes);
    if (e != cudaSuccess) return host_cuda_fail(e, "cudaMalloc(rounding sample)");
    do {
        if ((e = cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice)) != cudaSuccess) break;
        const int bs = 256, gs = (n + bs - 1) / bs;
        if (precision == RDC_F32_BF16STORE)
            k_sr_sample<__nv_bfloat16><<<gs, bs>>>(d, n, seed, step, row, col0, d + n, d + 2 * (size_t)n);
        else
            k_sr_sample<__half><<<gs, bs>>>(d, n, seed, step, row, col0, d + n, d + 2 * (size_t)n);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaMemcpy(u_out, d + n, bytes, cudaMemcpyDeviceToHost)) != cudaSuccess) break;
        e = cudaMemcpy(v_out, d + 2 * (size_t)n, bytes, cudaMemcpyDeviceToHost);
    } while (false);
    cudaFree(d);
    return e == cudaSuccess ? RDC_OK : host_cuda_fail(e, "rounding sample");
}

extern "C" int rdc_check_division(double q, uint64_t n_random, uint64_t seed,
                                  rdc_division_report* out)
{
    if (!out || !std::isfinite(q) || !(q > 0.0) || !(q < 1e30)) return RDC_EINVAL;
    int rc = host_check_device();
    if (rc) return rc;
    Counts* d = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return host_cuda_fail(e, "cudaStreamCreate");
    e = cudaMalloc((void**)&d, sizeof(Counts));
    if (e != cudaSuccess) {
        cudaStreamDestroy(st);
        return host_cuda_fail(e, "cudaMalloc(check counters)");
    }
    Counts h;
    for (int i = 0; i < 3; ++i) {
        h.checked[i] = h.bad[i] = 0;
        h.first_bad[i] = 0xffffffffu;
    }
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const dim3 grid(8 * (sms > 0 ? sms : 1)), block(256);
    do {
        if ((e = cudaMemcpyAsync(d, &h, sizeof(Counts), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            break;
        k_check_rcp<<<grid, block, 0, st>>>(d);
        k_check_ratio<<<grid, block, 0, st>>>((float)q, d);
        if (n_random) k_check_random<<<grid, block, 0, st>>>(n_random, seed, d);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(&h, d, sizeof(Counts), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            break;
        e = cudaStreamSynchronize(st);
    } while (false);
    cudaFree(d);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) return host_cuda_fail(e, "division check");
    for (int i = 0; i < 3; ++i) {
        out->checked[i] = h.checked[i];
        out->mismatches[i] = h.bad[i];
        out->first_bad[i] = h.first_bad[i];
    }
    return RDC_OK;
}
