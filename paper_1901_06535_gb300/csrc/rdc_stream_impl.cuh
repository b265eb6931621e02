// k_stepk_stream: K explicit Euler steps of Eq. 1 per launch (temporal
// blocking) with every intermediate time level held in registers.
//
// Each warp owns a strip of 32 * N columns (N cells per lane) and marches
// down a chunk of rows.  At iteration t it takes row t of u, v and phi (time
// level 0) and, for l = 1..K, computes row t - l of time level l from rows
// t-l-1, t-l, t-l+1 of level l-1 -- a wavefront in (row, time).  Each level
// keeps the last three u rows and two v rows it produced in registers, phi
// travels down the levels in a register queue, and only level K is written
// to memory.  East/west neighbours come from the adjacent lanes by shuffles,
// so a level is valid one column less on each side than the level before:
// warps overlap by HALO = roundup(K, N) columns per side (a multiple of N
// keeps every vector aligned) and each writes only its 32 * N - 2 * HALO
// interior columns.  Chunks overlap by K rows above and below for the same
// reason.  At the grid's own borders the mirror rule is applied either by
// selects in the level loop or, for the single-grid FP32 kernel at K >= 4,
// by loading the rows and columns beyond the border as mirror images.
//
// Per cell and level this does exactly what k_step1 does (same cell_update,
// same rounding to the storage type), so K steps here equal K launches of
// k_step1 bit for bit.  HBM traffic is that of one step per K steps (plus the
// halo overlap); the rest is FP32 (or FP64) arithmetic.
#pragma once

#include "rdc_device.cuh"
#include "rdc_internal.h"

namespace rdc {

// Unroll factor of the streamed kernel's row loop: the three-row register
// rotation and the K-deep phi queue become renaming when it is a multiple of
// both.  Measured at 8192^2 (A/B, identical bits), the single-grid FP32
// kernel with ghost cells (GH) runs best at K = 5 unrolled 5 times (809 -> 860
// G cell-updates/s; with the scalar horizontal sum 6 times lost 940 -> 913, 3
// times 898), K = 6 6 times (809 -> 852), K = 7 7 times (749 -> 771), K = 8 8
// times (735 -> 757), K = 4 6 times (12 lost 7 %).  The kernels with ghost
// cells (FP32 compute at K >= 4 without stochastic rounding, batched or not)
// take these; with border selects the batched FP32 kernel (UK) runs K = 6 six
// times (512-grid sweep: 813 -> 834) and the rest three times from K = 4.
template <int K, bool GH, bool UK>
constexpr int stream_unroll()
{
    if constexpr (GH) return K == 4 ? 6 : K;
    else if constexpr (UK && K == 6) return 6;
    else return K >= 4 ? 3 : 1;
}

// N consecutive stored values (N * sizeof(S) = 4, 8 or 16 bytes) -> compute
// type (S may also be a phi type: float or double).
template <typename S>
struct Widened { using T = typename Traits<S>::T; };

template <typename S, int N>
struct VecN {
    using T = typename Widened<S>::T;
    static constexpr int BYTES = N * (int)sizeof(S);
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "vector of 4, 8 or 16 bytes");
    union Raw {
        uint4 q;
        uint2 d;
        unsigned int w;
        S s[N];
    };
    static __device__ __forceinline__ void load(const S* p, T (&o)[N])
    {
        Raw r;
        if constexpr (BYTES == 16) r.q = __ldg(reinterpret_cast<const uint4*>(p));
        else if constexpr (BYTES == 8) r.d = __ldg(reinterpret_cast<const uint2*>(p));
        else r.w = __ldg(reinterpret_cast<const unsigned int*>(p));
#pragma unroll
        for (int e = 0; e < N; ++e) o[e] = widen(r.s[e]);
    }
    static __device__ __forceinline__ void store(S* p, const T (&x)[N])
    {
        Raw r;
#pragma unroll
        for (int e = 0; e < N; ++e) r.s[e] = narrow<S>(x[e]);
        if constexpr (BYTES == 16) *reinterpret_cast<uint4*>(p) = r.q;
        else if constexpr (BYTES == 8) *reinterpret_cast<uint2*>(p) = r.d;
        else *reinterpret_cast<unsigned int*>(p) = r.w;
    }
};

// Two values through the 16-bit storage type and back, one paired
// conversion each way (round to nearest even per value, as quantize).
template <typename S>
__device__ __forceinline__ float2 quantize2(float2 x);
template <>
__device__ __forceinline__ float2 quantize2<__nv_bfloat16>(float2 x)
{
    return __bfloat1622float2(__float22bfloat162_rn(x));
}
template <>
__device__ __forceinline__ float2 quantize2<__half>(float2 x)
{
    return __half22float2(__float22half2_rn(x));
}

// Mirror image of index x in [0, n) under the cell-centred zero-flux
// border: -1 -> 0, -2 -> 1, n -> n - 1, ... (repeated for grids narrower
// than the reach).
__device__ __forceinline__ int reflect_index(int x, int n)
{
    while (x < 0 || x >= n) x = (x < 0) ? -1 - x : 2 * n - 1 - x;
    return x;
}

// With stochastic rounding the overlap is a multiple of 4, so that every
// warp's first column starts a quad: with two cells per lane, lanes 2j and
// 2j + 1 then hold the two halves of one quad and share its random words.
template <typename S, int K, int N, bool SR = false>
struct StreamGeom {
    static constexpr int ALIGN = (SR && N < 4) ? 4 : N;
    static constexpr int HALO = (K + ALIGN - 1) / ALIGN * ALIGN;  // overlap per side, columns
    static constexpr int WCOLS = 32 * N;              // columns a warp holds
    static constexpr int OUTC = WCOLS - 2 * HALO;     // columns a warp writes
    static_assert(OUTC > 0, "halo wider than the warp");
};

// One warp's share: output columns [col_out, col_out + OUTC), output rows
// [y0, y1).  Warps are independent, so the same body serves one grid per
// launch (k_stepk_stream) and a work list over many grids (k_stream_batch).
//
// The row loop's body is straight-line code: every level computes its row
// even when that row lies outside the grid (garbage that no valid cell ever
// reads).  The mirror borders are applied either by selects (the select at
// rows 0 and H-1 and columns 0 and W-1 replaces the out-of-range neighbour by
// the cell itself) or, with GHOST, by loading the rows and columns beyond the
// border as mirror images.  phi of row t is loaded with row t's u and v and
// handed down the levels in a K-deep register queue (level l at iteration t
// needs row t - l), so each row's phi is read once; rows are loaded DIST
// iterations before their first use.  Straight-line code lets the compiler
// interleave the levels' arithmetic (warp-uniform branches in the level loop
// measured slower); the row loop is unrolled so that the three-row register
// rotation becomes renaming.
template <typename S, int MODE, int K, int N, bool GH, bool UK>
__device__ __forceinline__ void stream_warp_impl(const S* __restrict__ u,
                                                 const S* __restrict__ v,
                                                 const typename Traits<S>::PhiT* __restrict__ phi,
                                                 S* __restrict__ u1, S* __restrict__ v1, int W,
                                                 int H, int64_t pitch, int col_out, int y0,
                                                 int y1, const Model<typename Traits<S>::T>& m)
{
    using T = typename Traits<S>::T;
    using PhiT = typename Traits<S>::PhiT;
    using G = StreamGeom<S, K, N, (MODE & MODE_SR) != 0>;
    // GHOST: cells beyond the borders are loaded as mirror images of the cells
    // inside (rows and columns), so the level loop needs no border selects.
    // Addition is commutative, so a mirrored ghost cell evolves exactly like
    // its image and every valid cell gets the same bits as with the selects.
    // Not with stochastic rounding (a ghost would draw its own random bits).
    constexpr bool GHOST = GH && (MODE & MODE_SR) == 0;
    const int lane = threadIdx.x & 31;
    const int a = col_out - G::HALO;
    const int cl = a + lane * N;
    const bool in_grid = (cl >= 0) && (cl < W);
    const bool plain = (cl >= 0) && (cl + N <= W);  // every cell of the lane inside
    int srcc[N];                                     // mirrored source columns
#pragma unroll
    for (int e = 0; e < N; ++e) srcc[e] = reflect_index(cl + e, W);
    const int t0 = GHOST ? y0 - K : max(y0 - K, 0);
    const int t_end = y1 - 1 + K;
    // u, v, phi of row tl (mirrored rows and columns with GHOST; zeros outside
    // the grid otherwise)
    auto load_row = [&](int tl, T (&ru)[N], T (&rv)[N], T (&rp)[N]) {
        if constexpr (GHOST) {
            const int64_t ro = (int64_t)reflect_index(tl, H) * pitch;
            if (plain) {
                VecN<S, N>::load(u + ro + cl, ru);
                VecN<S, N>::load(v + ro + cl, rv);
                VecN<PhiT, N>::load(phi + ro + cl, rp);
            } else {
#pragma unroll
                for (int e = 0; e < N; ++e) {
                    ru[e] = widen(u[ro + srcc[e]]);
                    rv[e] = widen(v[ro + srcc[e]]);
                    rp[e] = (T)phi[ro + srcc[e]];
                }
            }
        } else if (tl < H && in_grid) {
            const int64_t o = (int64_t)tl * pitch + cl;
            VecN<S, N>::load(u + o, ru);
            VecN<S, N>::load(v + o, rv);
            VecN<PhiT, N>::load(phi + o, rp);
        }
    };
    T P0[K][N], P1[K][N], P2[K][N], Q0[K][N], Q1[K][N];
    T F[K][N];  // F[j]: phi of row t - 1 - j, loaded with that row's u and v
#pragma unroll
    for (int l = 0; l < K; ++l)
#pragma unroll
        for (int e = 0; e < N; ++e)
            P0[l][e] = P1[l][e] = P2[l][e] = Q0[l][e] = Q1[l][e] = F[l][e] = T(0);
    // Row t's u, v and phi are loaded DIST iterations ahead of their first use
    // (level 1 needs row t at once, and rows stream from HBM).  Measured at
    // 8192^2: one row ahead +25 % at K = 3 and +11 % at K = 6 (FP32); two rows
    // ahead another +6 % for the single-grid FP32 kernel at K >= 5 (GH; with
    // border selects it lost 9 % with 16-bit storage and 4 % in the batched
    // kernel, which now take the ghost cells and this distance with them);
    // none at K = 2, whose four cells per lane leave no registers (-14 %).
    constexpr int DIST = (GH && K >= 5) ? 2 : (K >= 3 ? 1 : 0);
    T pu[N], pv[N], pp[N], qu[N], qv[N], qp[N];
#pragma unroll
    for (int e = 0; e < N; ++e) pu[e] = pv[e] = pp[e] = qu[e] = qv[e] = qp[e] = T(0);
    if constexpr (DIST >= 1) load_row(t0, pu, pv, pp);
    if constexpr (DIST >= 2)
        if (t0 + 1 <= t_end) load_row(t0 + 1, qu, qv, qp);
    // Unrolled row loop: the three-row rotation becomes renaming; the kernels
    // with ghost cells at K = 4 (GH) run best unrolled six times (single-grid
    // FP32 835 vs 813 G cell-updates/s; with border selects six times lost
    // 17 % with 16-bit storage and 3 % in the batched kernel).
    constexpr int UNROLL = stream_unroll<K, GH, UK>();
#pragma unroll UNROLL
    for (int t = t0; t <= t_end; ++t) {
        T nphi[N];
        {
            T nu[N], nv[N];
#pragma unroll
            for (int e = 0; e < N; ++e) {
                nu[e] = pu[e];
                nv[e] = pv[e];
                nphi[e] = pp[e];
                if constexpr (DIST == 2) {
                    pu[e] = qu[e];
                    pv[e] = qv[e];
                    pp[e] = qp[e];
                    qu[e] = qv[e] = qp[e] = T(0);
                } else {
                    pu[e] = pv[e] = pp[e] = T(0);
                }
            }
            const int tl = t + DIST;  // the row loaded in this iteration
            if (tl <= t_end) {
                if constexpr (DIST == 2) load_row(tl, qu, qv, qp);
                else load_row(tl, pu, pv, pp);
            }
            if constexpr (DIST == 0) {
#pragma unroll
                for (int e = 0; e < N; ++e) {
                    nu[e] = pu[e];
                    nv[e] = pv[e];
                    nphi[e] = pp[e];
                }
            }
#pragma unroll
            for (int e = 0; e < N; ++e) {
                P2[0][e] = P1[0][e]; P1[0][e] = P0[0][e]; P0[0][e] = nu[e];
                Q1[0][e] = Q0[0][e]; Q0[0][e] = nv[e];
            }
        }
        unsigned wa = 0u, wb = 0u, wa_next = 0u, wb_next = 0u;  // shared random words
#pragma unroll
        for (int l = 1; l <= K; ++l) {
            const int r = t - l;
            const bool live = (r >= 0) && (r < H);   // warp-uniform
            T nu[N], nv[N];
            const T wsh = __shfl_up_sync(0xffffffffu, P1[l - 1][N - 1], 1);
            const T esh = __shfl_down_sync(0xffffffffu, P1[l - 1][0], 1);
            {
                const T (&ph)[N] = F[l - 1];
                const bool top = !GHOST && (r == 0), bottom = !GHOST && (r == H - 1);
                // stochastic rounding: the random words of the lane's cells
                // (wa, wb for N = 2; the whole quad rb for N = 4, whose lanes
                // start on multiples of 4).  With N = 2 the two lanes of a quad
                // share its Philox call in pairs of levels: for levels l, l + 1
                // the lane holding the quad's first half computes the quad's
                // words of level l, its partner those of level l + 1, and each
                // hands the other the two words it needs (a last odd level is
                // computed by both).
                const int rrow = r;
                Philox4 rb{0u, 0u, 0u, 0u};
                if constexpr ((MODE & MODE_SR) != 0 && N == 2) {
                    const bool second = (cl & 2) != 0;   // the quad's second half
                    if ((l & 1) == 1 && l < K) {
                        const Philox4 P = sr_quad_bits(m.seed, cl >> 2, second ? rrow - 1 : rrow,
                                                       m.step0 + l + (second ? 1 : 0));
                        const unsigned g0 = __shfl_xor_sync(0xffffffffu, second ? P.x : P.z, 1);
                        const unsigned g1 = __shfl_xor_sync(0xffffffffu, second ? P.y : P.w, 1);
                        wa = second ? g0 : P.x;
                        wb = second ? g1 : P.y;
                        wa_next = second ? P.z : g0;
                        wb_next = second ? P.w : g1;
                    } else if ((l & 1) == 0) {
                        wa = wa_next;
                        wb = wb_next;
                    } else {
                        const Philox4 P = sr_quad_bits(m.seed, cl >> 2, rrow, m.step0 + l);
                        wa = second ? P.z : P.x;
                        wb = second ? P.w : P.y;
                    }
                } else if constexpr ((MODE & MODE_SR) != 0) {
                    rb = sr_quad_bits(m.seed, cl >> 2, rrow, m.step0 + l);
                }
                if constexpr (sizeof(T) == 4 && N % 2 == 0) {
                    // FP32 compute: neighbouring cells in pairs (cell_update2).
                    // The border selects also assemble the west and east pairs.
#pragma unroll
                    for (int e = 0; e < N; e += 2) {
                        const int col = cl + e;
                        const float c0 = P1[l - 1][e], c1 = P1[l - 1][e + 1];
                        const float wr = (e == 0) ? wsh : P1[l - 1][e - 1];
                        const float er = (e + 2 == N) ? esh : P1[l - 1][e + 2];
                        const float2 c2 = make_float2(c0, c1);
                        const float2 w2 = make_float2(!GHOST && col <= 0 ? c0 : wr,
                                                      !GHOST && col + 1 <= 0 ? c1 : c0);
                        const float2 e2 = make_float2(!GHOST && col >= W - 1 ? c0 : c1,
                                                      !GHOST && col + 1 >= W - 1 ? c1 : er);
                        const float2 n2 = top ? c2 : make_float2(P2[l - 1][e], P2[l - 1][e + 1]);
                        const float2 s2 =
                            bottom ? c2 : make_float2(P0[l - 1][e], P0[l - 1][e + 1]);
                        float2 un, vn;
                        if constexpr (GHOST) {
                            // mirrored ghost cells (K >= 4): w + e as two
                            // scalar adds into an aligned pair, not a paired add
                            // of the pairs (w0, c0) and (c1, e1), which each need
                            // assembling by moves: the same bits, fewer registers
                            // and instructions (measured at 8192^2: K = 5 867 ->
                            // 934, K = 6 864 -> 945 G cell-updates/s; with it the
                            // batched kernel and the 16-bit storage kernels take
                            // the ghost cells too).  With border selects (K <= 3,
                            // stochastic rounding) the pairs are formed by the
                            // selects anyway and the paired add stays.
                            const float2 we2 = make_float2(__fadd_rn(w2.x, e2.x),
                                                           __fadd_rn(w2.y, e2.y));
                            cell_update2_we<MODE>(c2, we2, n2, s2,
                                                  make_float2(Q1[l - 1][e], Q1[l - 1][e + 1]),
                                                  make_float2(ph[e], ph[e + 1]), m, un, vn);
                        } else {
                            cell_update2<MODE>(c2, w2, e2, n2, s2,
                                               make_float2(Q1[l - 1][e], Q1[l - 1][e + 1]),
                                               make_float2(ph[e], ph[e + 1]), m, un, vn);
                        }
                        if constexpr ((MODE & MODE_SR) != 0) {
                            // stochastic rounding of level l (state step0 + l);
                            // BF16 by the add-and-carry form (sr_bf16), a NaN
                            // passed on as it is: it stays a NaN through the
                            // later levels and is stored as the canonical NaN,
                            // the bits the general form gives (a branch to the
                            // general form here would double the registers of
                            // the unrolled level loop)
                            unsigned w0, w1;
                            if constexpr (N == 2) {
                                w0 = wa;
                                w1 = wb;
                            } else {
                                const bool hi = (col & 2) != 0;  // words 2, 3 of the quad
                                w0 = hi ? rb.z : rb.x;
                                w1 = hi ? rb.w : rb.y;
                            }
                            if constexpr (std::is_same_v<S, __nv_bfloat16>) {
                                auto sr = [](float x, unsigned r16) {
                                    return isnan(x) ? x : sr_bf16(x, r16);
                                };
                                nu[e] = sr(un.x, w0 >> 16);
                                nu[e + 1] = sr(un.y, w1 >> 16);
                                nv[e] = sr(vn.x, w0 & 0xFFFFu);
                                nv[e + 1] = sr(vn.y, w1 & 0xFFFFu);
                            } else {
                                nu[e] = quantize_sr<S>(un.x, w0);
                                nu[e + 1] = quantize_sr<S>(un.y, w1);
                                nv[e] = quantize_sr<S>(vn.x, w0 << 16);
                                nv[e + 1] = quantize_sr<S>(vn.y, w1 << 16);
                            }
                        } else if constexpr (sizeof(S) == 2) {
                            const float2 qu = quantize2<S>(un), qv = quantize2<S>(vn);
                            nu[e] = qu.x;
                            nu[e + 1] = qu.y;
                            nv[e] = qv.x;
                            nv[e + 1] = qv.y;
                        } else {
                            nu[e] = quantize<S>(un.x);
                            nu[e + 1] = quantize<S>(un.y);
                            nv[e] = quantize<S>(vn.x);
                            nv[e + 1] = quantize<S>(vn.y);
                        }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < N; ++e) {
                        const int col = cl + e;
                        const T c = P1[l - 1][e];
                        T w = (e == 0) ? wsh : P1[l - 1][e - 1];
                        T ea = (e == N - 1) ? esh : P1[l - 1][e + 1];
                        if (!GHOST && col <= 0) w = c;
                        if (!GHOST && col >= W - 1) ea = c;
                        const T n = top ? c : P2[l - 1][e];
                        const T s = bottom ? c : P0[l - 1][e];
                        T un, vn;
                        cell_update<MODE>(c, w, ea, n, s, Q1[l - 1][e], ph[e], m, un, vn);
                        nu[e] = quantize<S>(un);
                        nv[e] = quantize<S>(vn);
                    }
                }
            }
            if (l < K) {
#pragma unroll
                for (int e = 0; e < N; ++e) {
                    P2[l][e] = P1[l][e]; P1[l][e] = P0[l][e]; P0[l][e] = nu[e];
                    Q1[l][e] = Q0[l][e]; Q0[l][e] = nv[e];
                }
            } else if (live && r >= y0 && r < y1) {
                if (cl >= col_out && cl < col_out + G::OUTC && cl < W) {
                    const int64_t o = (int64_t)r * pitch + cl;
                    if (cl + N <= W) {
                        VecN<S, N>::store(u1 + o, nu);
                        VecN<S, N>::store(v1 + o, nv);
                    } else {
#pragma unroll
                        for (int e = 0; e < N; ++e)
                            if (cl + e < W) { u1[o + e] = narrow<S>(nu[e]); v1[o + e] = narrow<S>(nv[e]); }
                    }
                }
            }
        }
#pragma unroll
        for (int j = K - 1; j > 0; --j)
#pragma unroll
            for (int e = 0; e < N; ++e) F[j][e] = F[j - 1][e];
#pragma unroll
        for (int e = 0; e < N; ++e) F[0][e] = nphi[e];
    }
}

template <typename S, int MODE, int K, int N, bool GH, bool UK = false>
__device__ __forceinline__ void stream_warp(const S* __restrict__ u, const S* __restrict__ v,
                                            const typename Traits<S>::PhiT* __restrict__ phi,
                                            S* __restrict__ u1, S* __restrict__ v1, int W,
                                            int H, int64_t pitch, int col_out, int y0, int y1,
                                            const Model<typename Traits<S>::T>& m)
{
    stream_warp_impl<S, MODE, K, N, GH, UK>(u, v, phi, u1, v1, W, H, pitch, col_out, y0, y1, m);
}

// The single-grid kernels at K >= 4 (GH) take the variants that measured
// faster there: mirrored ghost cells instead of border selects (FP32 K = 4:
// 724 -> 805, K = 6: 760 -> 786 G cell-updates/s at 8192^2), rows two
// iterations ahead at K >= 5 and a six-fold unroll at K = 4; they were slower
// for K <= 3, whose four cells per lane leave no registers.  16-bit storage
// takes them since the scalar horizontal sum freed its registers (BF16 K = 4
// 666 -> 720, K = 6 611 -> 698; FP16 703 -> 748, 644 -> 741); with stochastic
// rounding the ghost cells would draw random words of their own, so those
// kernels keep the border selects and their own unrolling.  The batched
// kernel takes them as well (stream_batch_body).  FP64 keeps the selects.
template <typename S, int MODE, int K>
constexpr bool stream_ghost()
{
    return sizeof(typename Traits<S>::T) == 4 && K >= 4 && (MODE & MODE_SR) == 0;
}

template <typename S, int MODE, int K, int N>
__device__ __forceinline__ void stepk_stream_body(const S* __restrict__ u, const S* __restrict__ v,
                                                  const typename Traits<S>::PhiT* __restrict__ phi,
                                                  S* __restrict__ u1, S* __restrict__ v1, int W,
                                                  int H, int64_t pitch, int rows, int nwarps_x,
                                                  const Model<typename Traits<S>::T>& m)
{
    using G = StreamGeom<S, K, N, (MODE & MODE_SR) != 0>;
    pdl_enter();
    const int wx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wx >= nwarps_x) return;                       // whole warps only
    const int y0 = blockIdx.y * rows;
    stream_warp<S, MODE, K, N, stream_ghost<S, MODE, K>()>(u, v, phi, u1, v1, W, H, pitch, wx * G::OUTC, y0,
                               min(y0 + rows, H), m);
}

template <typename S, int MODE, int K, int N>
__global__ void __launch_bounds__(128)
k_stepk_stream(const S* __restrict__ u, const S* __restrict__ v,
               const typename Traits<S>::PhiT* __restrict__ phi, S* __restrict__ u1,
               S* __restrict__ v1, int W, int H, int64_t pitch, int rows, int nwarps_x,
               Model<typename Traits<S>::T> m)
{
    stepk_stream_body<S, MODE, K, N>(u, v, phi, u1, v1, W, H, pitch, rows, nwarps_x, m);
}

// The same kernel with its registers capped so that MINB CTAs fit on an SM.
template <typename S, int MODE, int K, int N, int MINB>
__global__ void __launch_bounds__(128, MINB)
k_stepk_stream_capped(const S* __restrict__ u, const S* __restrict__ v,
                      const typename Traits<S>::PhiT* __restrict__ phi, S* __restrict__ u1,
                      S* __restrict__ v1, int W, int H, int64_t pitch, int rows, int nwarps_x,
                      Model<typename Traits<S>::T> m)
{
    stepk_stream_body<S, MODE, K, N>(u, v, phi, u1, v1, W, H, pitch, rows, nwarps_x, m);
}

// CTAs per SM the single-grid FP32 kernel is compiled for (0: the compiler's
// choice).  Measured at 8192^2 (A/B, identical bits), with the horizontal sum
// formed by scalar adds: K = 4 for 6 CTAs and K = 5 for 5 (78 and 92
// registers, no spill), K = 6 left at 94 registers (5 CTAs); K = 8 capped for 4
// (124 registers) 870 -> 895 G cell-updates/s; K = 5 for 6 (80 registers)
// lost 938 -> 877 and K = 6 for 5 lost 949 -> 900.
template <typename S, int MODE, int K>
constexpr int stream_single_min_ctas()
{
    return (sizeof(S) != 4 || (MODE & MODE_SR) != 0)
               ? 0
               : (K == 4 ? 6 : (K == 5 ? 5 : (K == 8 ? 4 : 0)));
}

// Persistent k-step launch over a batch of grids (see k_step1_batch).
template <typename S, int MODE, int K, int N>
__device__ __forceinline__ void stream_batch_body(const GridDesc* __restrict__ descs,
                                                  const TileMap* __restrict__ map, int rows,
                                                  unsigned* queue, int j, long long sbase)
{
    using T = typename Traits<S>::T;
    using PhiT = typename Traits<S>::PhiT;
    using G = StreamGeom<S, K, N, (MODE & MODE_SR) != 0>;
    pdl_enter();
    const int total = map->total;
    for (int it = queue_next(queue); it < total; it = queue_next(queue)) {
        int g, x0, y0;
        map_tile(map, it, G::OUTC, rows, g, x0, y0);
        const GridDesc& d = descs[g];
        const int par = (d.par + j) & 1;
        Model<T> m = model_of<T>(d);
        m.step0 += sbase;
        // mirrored ghost cells where the single-grid kernel takes them (with the
        // scalar horizontal sum they fit the register caps: the 512-grid FP32
        // sweep 834 -> 986 G cell-updates/s at K = 6; 128 grids at K = 6 with
        // BF16 storage 580 -> 616, FP16 589 -> 634)
        stream_warp<S, MODE, K, N, stream_ghost<S, MODE, K>(), sizeof(S) == 4>(
            static_cast<const S*>(d.u[par]), static_cast<const S*>(d.v[par]),
            static_cast<const PhiT*>(d.phi), static_cast<S*>(d.u[par ^ 1]),
            static_cast<S*>(d.v[par ^ 1]), d.W, d.H, d.pitch, x0, y0, min(y0 + rows, d.H), m);
    }
    queue_done(queue);
}

template <typename S, int MODE, int K, int N>
__global__ void __launch_bounds__(128)
k_stream_batch(const GridDesc* __restrict__ descs, const TileMap* __restrict__ map, int rows,
               unsigned* queue, int j, long long sbase)
{
    stream_batch_body<S, MODE, K, N>(descs, map, rows, queue, j, sbase);
}

// The same kernel with its registers capped so that MINB CTAs fit on an SM.
template <typename S, int MODE, int K, int N, int MINB>
__global__ void __launch_bounds__(128, MINB)
k_stream_batch_capped(const GridDesc* __restrict__ descs, const TileMap* __restrict__ map,
                      int rows, unsigned* queue, int j, long long sbase)
{
    stream_batch_body<S, MODE, K, N>(descs, map, rows, queue, j, sbase);
}

// CTAs per SM that the batched kernel is compiled for, 0 = the compiler's
// choice.  FP32 at K = 5 and 6 is capped at 6 and 5 CTAs (80 and 96
// registers instead of 92 and 111, no spills): measured on the 512-grid sweep,
// K = 5 793 -> 807 and K = 6 784 -> 827 G cell-updates/s, identical bits.  At
// K = 7 and 8 the same caps spill; an explicit cap of 1 elsewhere would change
// the compiler's allocation (K = 4: 72 -> 110 registers).
template <typename S, int K>
constexpr int batch_stream_min_ctas()
{
    return sizeof(S) != 4 ? 0 : (K == 5 ? 6 : (K == 6 ? 5 : 0));
}

// Cells per lane.  FP32 and 16-bit storage: 4 for K <= 3 (16-byte FP32
// vectors; 8-byte 16-bit u, v vectors), 2 for K >= 4, where the K levels'
// registers would otherwise cut the resident warps (measured: FP32 K = 4
// 489 -> 670 G cell-updates/s at 8192^2, BF16 storage K = 6 474 -> 550).
// FP64: 1.
template <typename S, int K>
struct StreamVec {
    static constexpr int N = (sizeof(S) == 8) ? 1 : (K <= 3 ? 4 : 2);
};

template <typename S, int K>
cudaError_t launch_stream_k(const Planes& g, const Model<typename Traits<S>::T>& m, int rows,
                            bool sr, cudaStream_t st)
{
    using PhiT = typename Traits<S>::PhiT;
    constexpr int N = StreamVec<S, K>::N;
    const int wpb = 4;  // warps per CTA (1 or 2 measured the same at K = 5, 6)
    if ((g.H + rows - 1) / rows > 65535) return cudaErrorInvalidValue;
    return dispatch_full<S>(sr, [&](auto mc) {
        using G = StreamGeom<S, K, N, (decltype(mc)::value & MODE_SR) != 0>;
        const int nwx = (g.W + G::OUTC - 1) / G::OUTC;
        const dim3 grid((nwx + wpb - 1) / wpb, (g.H + rows - 1) / rows);
        constexpr int MINB = stream_single_min_ctas<S, decltype(mc)::value, K>();
        if constexpr (MINB > 0)
            return launch_pdl(k_stepk_stream_capped<S, decltype(mc)::value, K, N, MINB>, grid,
                              dim3(32 * wpb), 0, st, static_cast<const S*>(g.u),
                              static_cast<const S*>(g.v), static_cast<const PhiT*>(g.phi),
                              static_cast<S*>(g.u1), static_cast<S*>(g.v1), g.W, g.H, g.pitch,
                              rows, nwx, m);
        else
            return launch_pdl(k_stepk_stream<S, decltype(mc)::value, K, N>, grid, dim3(32 * wpb),
                              0, st, static_cast<const S*>(g.u), static_cast<const S*>(g.v),
                              static_cast<const PhiT*>(g.phi), static_cast<S*>(g.u1),
                              static_cast<S*>(g.v1), g.W, g.H, g.pitch, rows, nwx, m);
    });
}

template <typename S, int K>
cudaError_t launch_stream_batch_k(const GridDesc* d, const TileMap* map, int rows,
                                  unsigned* queue, int j, long long sbase, bool sr, int ctas,
                                  cudaStream_t st)
{
    constexpr int N = StreamVec<S, K>::N;
    return dispatch_full<S>(sr, [&](auto mc) {
        constexpr int MINB = batch_stream_min_ctas<S, K>();
        if constexpr (MINB > 0)
            return launch_pdl(k_stream_batch_capped<S, decltype(mc)::value, K, N, MINB>,
                              dim3(ctas), dim3(128), 0, st, d, map, rows, queue, j, sbase);
        else
            return launch_pdl(k_stream_batch<S, decltype(mc)::value, K, N>, dim3(ctas),
                              dim3(128), 0, st, d, map, rows, queue, j, sbase);
    });
}

template <typename S>
cudaError_t launch_batch_stream_t(const GridDesc* d, const TileMap* map, int rows,
                                  unsigned* queue, int k, int j, long long sbase, int sr,
                                  int ctas, cudaStream_t st)
{
    if (ctas < 1 || rows < 1) return cudaErrorInvalidValue;
    const bool r = sr != 0;
    switch (k) {
        case 2: return launch_stream_batch_k<S, 2>(d, map, rows, queue, j, sbase, r, ctas, st);
        case 3: return launch_stream_batch_k<S, 3>(d, map, rows, queue, j, sbase, r, ctas, st);
        case 4: return launch_stream_batch_k<S, 4>(d, map, rows, queue, j, sbase, r, ctas, st);
        case 5: return launch_stream_batch_k<S, 5>(d, map, rows, queue, j, sbase, r, ctas, st);
        case 6: return launch_stream_batch_k<S, 6>(d, map, rows, queue, j, sbase, r, ctas, st);
        case 7: return launch_stream_batch_k<S, 7>(d, map, rows, queue, j, sbase, r, ctas, st);
        case 8: return launch_stream_batch_k<S, 8>(d, map, rows, queue, j, sbase, r, ctas, st);
    }
    return cudaErrorInvalidValue;
}

// Output columns per warp of the streamed kernel (sr: with stochastic
// rounding, whose overlap is a multiple of 4 columns).
template <typename S>
int stream_outc_t(int k, bool sr)
{
    switch (k) {
        case 2: return sr ? StreamGeom<S, 2, StreamVec<S, 2>::N, true>::OUTC : StreamGeom<S, 2, StreamVec<S, 2>::N>::OUTC;
        case 3: return sr ? StreamGeom<S, 3, StreamVec<S, 3>::N, true>::OUTC : StreamGeom<S, 3, StreamVec<S, 3>::N>::OUTC;
        case 4: return sr ? StreamGeom<S, 4, StreamVec<S, 4>::N, true>::OUTC : StreamGeom<S, 4, StreamVec<S, 4>::N>::OUTC;
        case 5: return sr ? StreamGeom<S, 5, StreamVec<S, 5>::N, true>::OUTC : StreamGeom<S, 5, StreamVec<S, 5>::N>::OUTC;
        case 6: return sr ? StreamGeom<S, 6, StreamVec<S, 6>::N, true>::OUTC : StreamGeom<S, 6, StreamVec<S, 6>::N>::OUTC;
        case 7: return sr ? StreamGeom<S, 7, StreamVec<S, 7>::N, true>::OUTC : StreamGeom<S, 7, StreamVec<S, 7>::N>::OUTC;
        case 8: return sr ? StreamGeom<S, 8, StreamVec<S, 8>::N, true>::OUTC : StreamGeom<S, 8, StreamVec<S, 8>::N>::OUTC;
    }
    return 0;
}

template <typename S>
cudaError_t launch_stream_t(const Planes& g, const ModelD& md, int k, int rows,
                            cudaStream_t st)
{
    if (rows < 1) return cudaErrorInvalidValue;
    auto m = make_model<S>(md);
    const bool sr = md.sr != 0;
    switch (k) {
        case 2: return launch_stream_k<S, 2>(g, m, rows, sr, st);
        case 3: return launch_stream_k<S, 3>(g, m, rows, sr, st);
        case 4: return launch_stream_k<S, 4>(g, m, rows, sr, st);
        case 5: return launch_stream_k<S, 5>(g, m, rows, sr, st);
        case 6: return launch_stream_k<S, 6>(g, m, rows, sr, st);
        case 7: return launch_stream_k<S, 7>(g, m, rows, sr, st);
        case 8: return launch_stream_k<S, 8>(g, m, rows, sr, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace rdc
