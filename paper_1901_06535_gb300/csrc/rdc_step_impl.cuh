// Step kernels of the Oregonator model (Eq. 1, explicit Euler, five-node
// Laplacian with zero-flux borders, §2).  Included once per storage type by
// rdc_step_<type>.cu so the precisions compile in parallel.
//
//  k_step1 : one Euler step per launch.  HBM-bound: per cell it reads u, v,
//            phi once and writes u', v' once.  Each thread owns one 16-byte
//            vector of cells in a row and marches down `rows` rows, keeping
//            the north / centre / south rows of u in registers, so u is read
//            from memory once; east/west neighbours across vector edges come
//            from warp shuffles, and only the two cells beyond each warp's
//            span are loaded separately.  FP32-compute cells go in pairs
//            (cell_update2); consecutive launches alternate the row order so
//            each step starts on rows still in L2.
//  k_stepk : k Euler steps per launch (temporal blocking).  A CTA loads a
//            (tx + 2k) x (ty + 2k) tile of u, v, phi into shared memory and
//            steps it k times, the valid region shrinking by one cell per
//            side per step (ghost-zone recompute), then writes the tx x ty
//            interior.  Each intermediate u, v is rounded to the storage type
//            exactly as k_step1 stores it, so k launches of k_step1 and one
//            launch of k_stepk give the same bits.
#pragma once

#include <mutex>
#include <type_traits>

#include "rdc_device.cuh"
#include "rdc_internal.h"

namespace rdc {

// Calls f(std::integral_constant<int, MODE>) for the step kernel's template
// mode: the physics mode, plus MODE_SR with stochastic rounding, which only
// the 16-bit storage types instantiate.
template <typename S, int M, typename F>
cudaError_t call_mode(F&& f)
{
    if constexpr ((M & MODE_SR) != 0 && sizeof(S) != 2) return cudaErrorInvalidValue;
    else return f(std::integral_constant<int, M>{});
}

// The full model only (streamed and batched kernels).
template <typename S, typename F>
cudaError_t dispatch_full(bool sr, F&& f)
{
    return sr ? call_mode<S, MODE_FULL | MODE_SR>(f) : call_mode<S, MODE_FULL>(f);
}

template <typename S, typename F>
cudaError_t dispatch_mode(int mode, bool sr, F&& f)
{
    switch (mode) {
        case MODE_FULL:
            return sr ? call_mode<S, MODE_FULL | MODE_SR>(f) : call_mode<S, MODE_FULL>(f);
        case MODE_DIFFUSION:
            return sr ? call_mode<S, MODE_DIFFUSION | MODE_SR>(f) : call_mode<S, MODE_DIFFUSION>(f);
        case MODE_REACTION:
            return sr ? call_mode<S, MODE_REACTION | MODE_SR>(f) : call_mode<S, MODE_REACTION>(f);
    }
    return cudaErrorInvalidValue;
}

// VEC stored values from p: one 16-byte vector (Vec<S>), or, for a BF16 quad,
// one 8-byte vector.
template <typename S, int VEC>
__device__ __forceinline__ void vload(const S* p, typename Traits<S>::T (&o)[VEC], bool stream)
{
    if constexpr (VEC == Traits<S>::VEC) {
        if (stream) Vec<S>::load_stream(p, o);
        else Vec<S>::load(p, o);
    } else {
        static_assert(sizeof(S) == 2 && VEC == 4, "a quad of 16-bit cells");
        const uint2 r = stream ? __ldcs(reinterpret_cast<const uint2*>(p))
                               : __ldg(reinterpret_cast<const uint2*>(p));
        float2 a, b;
        if constexpr (std::is_same_v<S, __nv_bfloat16>) {
            a = bf2_to_f2(r.x);
            b = bf2_to_f2(r.y);
        } else {
            a = h2_to_f2(r.x);
            b = h2_to_f2(r.y);
        }
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
}

// Cells per lane of the single-step kernel: one 16-byte vector (with
// stochastic rounding two quads, computed and rounded one after the other).
// One quad (8 bytes) per lane was tried for stochastic rounding to leave room
// for more resident warps; at 8192^2 the 16-byte vectors at 72 registers are
// faster (BF16 399 -> 416, FP16 363 -> 397 G cell-updates/s, identical bits).
template <typename S, int MODE>
constexpr int step1_vec()
{
    return Traits<S>::VEC;
}

// One row of a lane's VEC cells (VEC / 4 whole quads) of a single Euler step
// under stochastic rounding: the cell updates from the north, centre and south
// rows of u (un, uc, us; wl, er: the cells west and east of the lane's span),
// v and phi of the row, then u' and v' of row r rounded stochastically to S
// and stored at ro + col0.  16-bit storage, one quad at a time -- its two cell
// pairs, its random words, its rounding, its packed words -- so that only one
// quad's values are live at once.  BF16 takes the add-and-carry form of the
// rule (sr_bf16; the packed words take the upper halves of the sums directly)
// unless the quad holds a NaN, which the paired sum of its values exposes (an
// infinity of each sign also sends the quad to the general form, which is
// exact for every value); FP16 takes it (sr_f16_normal) when all eight values
// lie in FP16's normal range, else the general form.
template <typename S, int MODE, int VEC>
__device__ __forceinline__ void sr_row(const float (&un)[VEC], const float (&uc)[VEC],
                                       const float (&us)[VEC], const float (&vv)[VEC],
                                       const float (&ph)[VEC], float wl, float er, int col0,
                                       int W, int r, int64_t ro, S* __restrict__ u1,
                                       S* __restrict__ v1, const Model<float>& m)
{
    static_assert(sizeof(S) == 2 && VEC % 4 == 0, "16-bit storage, whole quads");
    unsigned pu[VEC / 2], pv[VEC / 2];
#pragma unroll
    for (int e = 0; e < VEC; e += 4) {
        float2 a2, b2, c2, d2;   // u', v' of cells e, e+1 and e+2, e+3
#pragma unroll
        for (int h = 0; h < 4; h += 2) {
            const int x = e + h;
            const float c0 = uc[x], c1 = uc[x + 1];
            const float2 w2 = make_float2((x == 0) ? wl : uc[x - 1], c0);
            const float2 e2 = make_float2(col0 + x >= W - 1 ? c0 : c1,
                                          col0 + x + 1 >= W - 1
                                              ? c1
                                              : ((x + 2 == VEC) ? er : uc[x + 2]));
            cell_update2<MODE>(make_float2(c0, c1), w2, e2,
                               make_float2(un[x], un[x + 1]),
                               make_float2(us[x], us[x + 1]),
                               make_float2(vv[x], vv[x + 1]),
                               make_float2(ph[x], ph[x + 1]), m, h ? c2 : a2,
                               h ? d2 : b2);
        }
        const Philox4 rb = sr_quad_bits(m.seed, (col0 + e) >> 2, r, m.step0 + 1);
        const float2 chk = __fadd2_rn(__fadd2_rn(a2, b2), __fadd2_rn(c2, d2));
        const unsigned w[4] = {rb.x, rb.y, rb.z, rb.w};
        auto pack = [](float a, float b) {
            if constexpr (std::is_same_v<S, __nv_bfloat16>) return f2_to_bf2(a, b);
            else return f2_to_h2(a, b);
        };
        if (std::is_same_v<S, __nv_bfloat16> && !(isnan(chk.x) || isnan(chk.y))) {
            pu[e / 2] = pack_upper(sr_bf16_carry(a2.x, w[0] >> 16),
                                   sr_bf16_carry(a2.y, w[1] >> 16));
            pu[e / 2 + 1] = pack_upper(sr_bf16_carry(c2.x, w[2] >> 16),
                                       sr_bf16_carry(c2.y, w[3] >> 16));
            pv[e / 2] = pack_upper(sr_bf16_carry(b2.x, w[0] & 0xFFFFu),
                                   sr_bf16_carry(b2.y, w[1] & 0xFFFFu));
            pv[e / 2 + 1] = pack_upper(sr_bf16_carry(d2.x, w[2] & 0xFFFFu),
                                       sr_bf16_carry(d2.y, w[3] & 0xFFFFu));
        } else if (std::is_same_v<S, __half> &&
                   fp16_normal(a2.x) && fp16_normal(a2.y) && fp16_normal(b2.x) &&
                   fp16_normal(b2.y) && fp16_normal(c2.x) && fp16_normal(c2.y) &&
                   fp16_normal(d2.x) && fp16_normal(d2.y)) {
            pu[e / 2] = pack(sr_f16_normal(a2.x, w[0] >> 16),
                             sr_f16_normal(a2.y, w[1] >> 16));
            pu[e / 2 + 1] = pack(sr_f16_normal(c2.x, w[2] >> 16),
                                 sr_f16_normal(c2.y, w[3] >> 16));
            pv[e / 2] = pack(sr_f16_normal(b2.x, w[0] & 0xFFFFu),
                             sr_f16_normal(b2.y, w[1] & 0xFFFFu));
            pv[e / 2 + 1] = pack(sr_f16_normal(d2.x, w[2] & 0xFFFFu),
                                 sr_f16_normal(d2.y, w[3] & 0xFFFFu));
        } else {
            pu[e / 2] = pack(quantize_sr<S>(a2.x, w[0]), quantize_sr<S>(a2.y, w[1]));
            pu[e / 2 + 1] = pack(quantize_sr<S>(c2.x, w[2]), quantize_sr<S>(c2.y, w[3]));
            pv[e / 2] = pack(quantize_sr<S>(b2.x, w[0] << 16),
                             quantize_sr<S>(b2.y, w[1] << 16));
            pv[e / 2 + 1] = pack(quantize_sr<S>(d2.x, w[2] << 16),
                                 quantize_sr<S>(d2.y, w[3] << 16));
        }
    }
    if (col0 + VEC <= W) {
        if constexpr (VEC == 8) {
            st16(u1 + ro + col0, make_uint4(pu[0], pu[1], pu[2], pu[3]));
            st16(v1 + ro + col0, make_uint4(pv[0], pv[1], pv[2], pv[3]));
        } else {
            *reinterpret_cast<uint2*>(u1 + ro + col0) = make_uint2(pu[0], pu[1]);
            *reinterpret_cast<uint2*>(v1 + ro + col0) = make_uint2(pv[0], pv[1]);
        }
    } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            if (col0 + e < W) {
                const int sh = 16 * (e & 1);
                const unsigned short hu = (unsigned short)(pu[e / 2] >> sh);
                const unsigned short hv = (unsigned short)(pv[e / 2] >> sh);
                if constexpr (std::is_same_v<S, __nv_bfloat16>) {
                    u1[ro + col0 + e] = __ushort_as_bfloat16(hu);
                    v1[ro + col0 + e] = __ushort_as_bfloat16(hv);
                } else {
                    u1[ro + col0 + e] = __ushort_as_half(hu);
                    v1[ro + col0 + e] = __ushort_as_half(hv);
                }
            }
        }
    }
}

// One warp's share of a single Euler step: 32 vectors of VEC cells starting
// at column wcol0, rows [row0, row1).  Warps are independent (no shared
// memory, no block barrier), so the same body serves one grid per launch
// (k_step1) and a work list over many grids (k_step1_batch).
template <typename S, int MODE, int VEC = Traits<S>::VEC>
__device__ __forceinline__ void step1_warp(const S* __restrict__ u, const S* __restrict__ v,
                                           const typename Traits<S>::PhiT* __restrict__ phi,
                                           S* __restrict__ u1, S* __restrict__ v1, int W,
                                           int H, int64_t pitch, int wcol0, int row0,
                                           int row1, const Model<typename Traits<S>::T>& m)
{
    using T = typename Traits<S>::T;
    const int lane = threadIdx.x & 31;
    const int col0 = wcol0 + lane * VEC;
    const bool act = col0 < W;

    T un[VEC], uc[VEC], us[VEC], vv[VEC], ph[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) un[e] = uc[e] = us[e] = vv[e] = ph[e] = T(0);

    if (act) {
        vload<S, VEC>(u + (int64_t)max(row0 - 1, 0) * pitch + col0, un, false);
        vload<S, VEC>(u + (int64_t)row0 * pitch + col0, uc, false);
    }
    for (int r = row0; r < row1; ++r) {
        const int64_t ro = (int64_t)r * pitch;
        const int64_t rso = (int64_t)min(r + 1, H - 1) * pitch;
        T wl = T(0), er = T(0);
        if (act) {
            vload<S, VEC>(u + rso + col0, us, false);
            vload<S, VEC>(v + ro + col0, vv, true);
            load_phi<VEC>(phi + ro + col0, ph);
            if (lane == 0) wl = (col0 > 0) ? widen(u[ro + col0 - 1]) : uc[0];
            if (lane == 31 && col0 + VEC < W) er = widen(u[ro + col0 + VEC]);
        }
        const T wsh = __shfl_up_sync(0xffffffffu, uc[VEC - 1], 1);
        const T esh = __shfl_down_sync(0xffffffffu, uc[0], 1);
        if (lane != 0) wl = wsh;
        if (lane != 31) er = esh;
        if constexpr ((MODE & MODE_SR) != 0) {
            if (act) sr_row<S, MODE, VEC>(un, uc, us, vv, ph, wl, er, col0, W, r, ro, u1, v1, m);
        } else if (act) {
            static_assert(VEC == Traits<S>::VEC, "16-byte vectors outside the stochastic rounding path");
            T ou[VEC], ov[VEC];
            if constexpr (sizeof(T) == 4) {
                // FP32 compute: neighbouring cells in pairs (cell_update2)
#pragma unroll
                for (int e = 0; e < VEC; e += 2) {
                    const float c0 = uc[e], c1 = uc[e + 1];
                    const float2 w2 = make_float2((e == 0) ? wl : uc[e - 1], c0);
                    const float2 e2 = make_float2(col0 + e >= W - 1 ? c0 : c1,
                                                  col0 + e + 1 >= W - 1
                                                      ? c1
                                                      : ((e + 2 == VEC) ? er : uc[e + 2]));
                    float2 o2, p2;
                    cell_update2<MODE>(make_float2(c0, c1), w2, e2, make_float2(un[e], un[e + 1]),
                                       make_float2(us[e], us[e + 1]),
                                       make_float2(vv[e], vv[e + 1]),
                                       make_float2(ph[e], ph[e + 1]), m, o2, p2);
                    ou[e] = o2.x;
                    ou[e + 1] = o2.y;
                    ov[e] = p2.x;
                    ov[e + 1] = p2.y;
                }
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const T w = (e == 0) ? wl : uc[e - 1];
                    T ea = (e == VEC - 1) ? er : uc[e + 1];
                    if (col0 + e >= W - 1) ea = uc[e];  // mirror at the east border
                    cell_update<MODE>(uc[e], w, ea, un[e], us[e], vv[e], ph[e], m, ou[e], ov[e]);
                }
            }
            if (col0 + VEC <= W) {
                Vec<S>::store(u1 + ro + col0, ou);
                Vec<S>::store(v1 + ro + col0, ov);
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    if (col0 + e < W) {
                        u1[ro + col0 + e] = narrow<S>(ou[e]);
                        v1[ro + col0 + e] = narrow<S>(ov[e]);
                    }
                }
            }
        }
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            un[e] = uc[e];
            uc[e] = us[e];
        }
    }
}

// Register cap: at most 72 registers, so that the 16-bit-storage
// instantiations (8 cells per thread) fit 7 CTAs per SM, with stochastic
// rounding too (BF16 spills 76 bytes there and is still faster than at 80 or
// 96 registers: 416 against 406 and 386 G cell-updates/s at 8192^2).
template <typename S, int MODE>
constexpr int step1_max_regs()
{
    return 72;
}

template <typename S, int MODE>
__global__ void __maxnreg__((step1_max_regs<S, MODE>()))
k_step1(const S* __restrict__ u, const S* __restrict__ v,
        const typename Traits<S>::PhiT* __restrict__ phi, S* __restrict__ u1,
        S* __restrict__ v1, int W, int H, int64_t pitch, int rows,
        Model<typename Traits<S>::T> m, int flip)
{
    constexpr int VEC = step1_vec<S, MODE>();
    pdl_enter();
    const int wcol0 = (blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * VEC;
    // Consecutive launches sweep the rows in opposite directions (flip), so a
    // step starts on the rows the previous step wrote last, which are still
    // in L2: measured 340 -> 347 G cell-updates/s at 8192^2 (FP32), +3 % with
    // 16-bit storage.  The order does not change any result (Jacobi update).
    const int by = flip ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y;
    const int row0 = by * rows;
    step1_warp<S, MODE, VEC>(u, v, phi, u1, v1, W, H, pitch, wcol0, row0, min(row0 + rows, H),
                             m);
}

template <typename T>
__device__ __forceinline__ Model<T> model_of(const GridDesc& d)
{
    Model<T> m;
    m.eps = (T)d.eps;
    m.f = (T)d.f;
    m.q = (T)d.q;
    m.Du = (T)d.Du;
    m.dt = (T)d.dt;
    m.inv_dx2 = (T)d.inv_dx2;
    m.dt_Dux = (T)(__dmul_rn(__dmul_rn(d.dt, d.Du), d.inv_dx2));
    m.dt_eps = (T)(__ddiv_rn(d.dt, d.eps));
    m.seed = d.seed;
    m.step0 = d.steps;
    return m;
}

// Persistent single step over a batch of grids: every warp takes tiles from
// the work queue until the map is exhausted; a tile is one warp's strip of
// 32 vectors of one grid.
template <typename S, int MODE>
__global__ void __launch_bounds__(128)
k_step1_batch(const GridDesc* __restrict__ descs, const TileMap* __restrict__ map, int rows,
              unsigned* queue, int j, long long sbase)
{
    using T = typename Traits<S>::T;
    using PhiT = typename Traits<S>::PhiT;
    constexpr int COLS = 32 * Traits<S>::VEC;
    pdl_enter();
    const int total = map->total;
    for (int it = queue_next(queue); it < total; it = queue_next(queue)) {
        int g, x0, y0;
        map_tile(map, it, COLS, rows, g, x0, y0);
        const GridDesc& d = descs[g];
        const int par = (d.par + j) & 1;
        Model<T> m = model_of<T>(d);
        m.step0 += sbase;
        step1_warp<S, MODE>(static_cast<const S*>(d.u[par]), static_cast<const S*>(d.v[par]),
                            static_cast<const PhiT*>(d.phi), static_cast<S*>(d.u[par ^ 1]),
                            static_cast<S*>(d.v[par ^ 1]), d.W, d.H, d.pitch, x0, y0,
                            min(y0 + rows, d.H), m);
    }
    queue_done(queue);
}

template <typename S>
cudaError_t launch_batch_step1_t(const GridDesc* d, const TileMap* map, int rows,
                                 unsigned* queue, int j, long long sbase, int sr, int ctas,
                                 cudaStream_t st)
{
    if (ctas < 1 || rows < 1) return cudaErrorInvalidValue;
    return dispatch_full<S>(sr != 0, [&](auto mc) {
        return launch_pdl(k_step1_batch<S, decltype(mc)::value>, dim3(ctas), dim3(128), 0, st, d,
                          map, rows, queue, j, sbase);
    });
}

// Shared-memory layout of k_stepk: four planes of (tx+2k) x (ty+2k) compute
// values: u (ping), u (pong), v (updated in place: v' of a cell depends only
// on that cell), phi.
template <typename S, int MODE>
__global__ void __launch_bounds__(512)
k_stepk(const S* __restrict__ u, const S* __restrict__ v,
        const typename Traits<S>::PhiT* __restrict__ phi, S* __restrict__ u1,
        S* __restrict__ v1, int W, int H, int64_t pitch, int TX, int TY, int K,
        Model<typename Traits<S>::T> m)
{
    using T = typename Traits<S>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int RX = TX + 2 * K, RY = TY + 2 * K;
    const int area = RX * RY;
    T* ua = reinterpret_cast<T*>(smem_raw);
    T* ub = ua + area;
    T* vs = ub + area;
    T* ps = vs + area;

    const int gx0 = blockIdx.x * TX - K;  // global column of local column 0
    const int gy0 = blockIdx.y * TY - K;  // global row of local row 0
    const int nt = blockDim.x;
    const int tid = threadIdx.x;

    // load the tile (cells outside the grid are never read)
    for (int idx = tid; idx < area; idx += nt) {
        const int ly = idx / RX, lx = idx - ly * RX;
        const int gy = gy0 + ly, gx = gx0 + lx;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            const int64_t o = (int64_t)gy * pitch + gx;
            ua[idx] = widen(u[o]);
            vs[idx] = widen(v[o]);
            ps[idx] = (T)phi[o];
        }
    }
    __syncthreads();

    const int lane = tid & 31, wy = tid >> 5, nwy = nt >> 5;
    T* cur = ua;
    T* nxt = ub;
    for (int s = 1; s <= K; ++s) {
        const int ylo = max(s, -gy0), yhi = min(RY - s, H - gy0);
        const int xlo = max(s, -gx0), xhi = min(RX - s, W - gx0);
        for (int ly = ylo + wy; ly < yhi; ly += nwy) {
            const int gy = gy0 + ly;
            const int rowo = ly * RX;
            const int no = (gy > 0) ? -RX : 0;
            const int so = (gy < H - 1) ? RX : 0;
            for (int lx = xlo + lane; lx < xhi; lx += 32) {
                const int gx = gx0 + lx;
                const int i = rowo + lx;
                const T c = cur[i];
                const T w = (gx > 0) ? cur[i - 1] : c;
                const T e = (gx < W - 1) ? cur[i + 1] : c;
                const T n = cur[i + no];
                const T so_v = cur[i + so];
                T un, vn;
                cell_update<MODE>(c, w, e, n, so_v, vs[i], ps[i], m, un, vn);
                if constexpr ((MODE & MODE_SR) != 0) {
                    const unsigned w =
                        sr_word(sr_quad_bits(m.seed, gx >> 2, gy, m.step0 + s), gx & 3);
                    nxt[i] = quantize_sr<S>(un, w);
                    vs[i] = quantize_sr<S>(vn, w << 16);
                } else {
                    nxt[i] = quantize<S>(un);
                    vs[i] = quantize<S>(vn);
                }
            }
        }
        __syncthreads();
        T* t = cur;
        cur = nxt;
        nxt = t;
    }

    // write the interior
    for (int idx = tid; idx < TX * TY; idx += nt) {
        const int iy = idx / TX, ix = idx - iy * TX;
        const int gy = gy0 + K + iy, gx = gx0 + K + ix;
        if (gy < H && gx < W) {
            const int i = (iy + K) * RX + (ix + K);
            const int64_t o = (int64_t)gy * pitch + gx;
            u1[o] = narrow<S>(cur[i]);
            v1[o] = narrow<S>(vs[i]);
        }
    }
}

template <typename S>
Model<typename Traits<S>::T> make_model(const ModelD& d)
{
    using T = typename Traits<S>::T;
    Model<T> m;
    m.eps = (T)d.eps;
    m.f = (T)d.f;
    m.q = (T)d.q;
    m.Du = (T)d.Du;
    m.dt = (T)d.dt;
    m.inv_dx2 = (T)d.inv_dx2;
    m.dt_Dux = (T)((d.dt * d.Du) * d.inv_dx2);
    m.dt_eps = (T)(d.dt / d.eps);
    m.seed = d.seed;
    m.step0 = d.step0;
    return m;
}

template <typename S>
cudaError_t launch_step1_t(int mode, const Planes& g, const ModelD& md, Shape1 sh,
                           cudaStream_t st)
{
    using PhiT = typename Traits<S>::PhiT;
    if (sh.bx < 32 || sh.bx > 256 || (sh.bx % 32) != 0 || sh.rows < 1)
        return cudaErrorInvalidValue;
    int rows = sh.rows;
    if ((g.H + rows - 1) / rows > 65535) rows = (g.H + 65534) / 65535;
    auto m = make_model<S>(md);
    const S* u = static_cast<const S*>(g.u);
    const S* v = static_cast<const S*>(g.v);
    const PhiT* phi = static_cast<const PhiT*>(g.phi);
    S* u1 = static_cast<S*>(g.u1);
    S* v1 = static_cast<S*>(g.v1);
    const dim3 block(sh.bx);
    return dispatch_mode<S>(mode, md.sr != 0, [&](auto mc) {
        constexpr int VEC = step1_vec<S, decltype(mc)::value>();
        const int vecs = (g.W + VEC - 1) / VEC;
        const dim3 grid((vecs + sh.bx - 1) / sh.bx, (g.H + rows - 1) / rows);
        return launch_pdl(k_step1<S, decltype(mc)::value>, grid, block, 0, st, u, v, phi, u1, v1,
                          g.W, g.H, g.pitch, rows, m, md.flip);
    });
}

template <typename S>
size_t stepk_smem_t(ShapeK s)
{
    using T = typename Traits<S>::T;
    return (size_t)4 * (s.tx + 2 * s.k) * (s.ty + 2 * s.k) * sizeof(T);
}

template <typename S, int MODE>
cudaError_t set_stepk_attr(size_t smem)
{
    // Largest dynamic shared memory already granted, per device, per
    // instantiation; raised monotonically, under a lock (separate handles may
    // launch from several threads at once).
    static size_t configured[64] = {0};
    static std::mutex mu;
    if (smem <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (smem > configured[dev]) {
        e = cudaFuncSetAttribute(k_stepk<S, MODE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev] = smem;
    }
    return cudaSuccess;
}

template <typename S>
cudaError_t launch_stepk_t(int mode, const Planes& g, const ModelD& md, ShapeK sh,
                           cudaStream_t st)
{
    using PhiT = typename Traits<S>::PhiT;
    if (sh.k < 1 || sh.k > 8 || sh.tx < 1 || sh.ty < 1 || sh.nthreads < 32 ||
        sh.nthreads > 512 || (sh.nthreads % 32) != 0)
        return cudaErrorInvalidValue;
    const size_t smem = stepk_smem_t<S>(sh);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    dim3 grid((g.W + sh.tx - 1) / sh.tx, (g.H + sh.ty - 1) / sh.ty);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    auto m = make_model<S>(md);
    const S* u = static_cast<const S*>(g.u);
    const S* v = static_cast<const S*>(g.v);
    const PhiT* phi = static_cast<const PhiT*>(g.phi);
    S* u1 = static_cast<S*>(g.u1);
    S* v1 = static_cast<S*>(g.v1);
    cudaError_t e = dispatch_mode<S>(mode, md.sr != 0, [&](auto mc) {
        constexpr int M = decltype(mc)::value;
        cudaError_t ea = set_stepk_attr<S, M>(smem);
        if (ea != cudaSuccess) return ea;
        k_stepk<S, M><<<grid, sh.nthreads, smem, st>>>(u, v, phi, u1, v1, g.W, g.H, g.pitch,
                                                        sh.tx, sh.ty, sh.k, m);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace rdc
