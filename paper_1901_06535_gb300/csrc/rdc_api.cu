// C ABI of librdc (include/rdc.h): handles, validation, memory layout,
// dispatch of the step kernels, host <-> device transfers.
//
// Device layout of a library-owned simulation: one allocation holding
//   u[0], u[1], v[0], v[1]  (storage type, ping-pong),  phi  (float, or
//   double in FP64 mode),  then a small scratch area (health flag, probe
//   buffers);
// every plane is row-major with a row pitch of roundup(W, 64) elements, so
// each row starts on a 128-byte boundary and 16-byte vector accesses of any
// storage type stay aligned.  Plane offsets are multiples of 256 bytes.
#include <algorithm>
#include <climits>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rdc.h"
#include "rdc_host.h"
#include "rdc_internal.h"

static nvtxDomainHandle_t nvtx_domain()
{
    static nvtxDomainHandle_t d = nvtxDomainCreateA("librdc");
    return d;
}

NvtxRange::NvtxRange(const char* name)
{
    nvtxEventAttributes_t a = {};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    nvtxDomainRangePushEx(nvtx_domain(), &a);
}

NvtxRange::~NvtxRange() { nvtxDomainRangePop(nvtx_domain()); }

namespace rdc {
cudaError_t launch_step1_f32(int, const Planes&, const ModelD&, Shape1, cudaStream_t);
cudaError_t launch_step1_f64(int, const Planes&, const ModelD&, Shape1, cudaStream_t);
cudaError_t launch_step1_bf16(int, const Planes&, const ModelD&, Shape1, cudaStream_t);
cudaError_t launch_step1_f16(int, const Planes&, const ModelD&, Shape1, cudaStream_t);
cudaError_t launch_stepk_f32(int, const Planes&, const ModelD&, ShapeK, cudaStream_t);
cudaError_t launch_stepk_f64(int, const Planes&, const ModelD&, ShapeK, cudaStream_t);
cudaError_t launch_stepk_bf16(int, const Planes&, const ModelD&, ShapeK, cudaStream_t);
cudaError_t launch_stepk_f16(int, const Planes&, const ModelD&, ShapeK, cudaStream_t);
size_t stepk_smem_f32(ShapeK);
size_t stepk_smem_f64(ShapeK);
size_t stepk_smem_bf16(ShapeK);
size_t stepk_smem_f16(ShapeK);
cudaError_t launch_stream_f32(const Planes&, const ModelD&, int, int, cudaStream_t);
cudaError_t launch_stream_f64(const Planes&, const ModelD&, int, int, cudaStream_t);
cudaError_t launch_stream_bf16(const Planes&, const ModelD&, int, int, cudaStream_t);
cudaError_t launch_stream_f16(const Planes&, const ModelD&, int, int, cudaStream_t);
#define RDC_DECL_BATCH(n)                                                                   \
    cudaError_t launch_batch_step1_##n(const GridDesc*, const TileMap*, int, unsigned*, int,   \
                                       long long, int, int, cudaStream_t);                  \
    cudaError_t launch_batch_stream_##n(const GridDesc*, const TileMap*, int, unsigned*, int,  \
                                        int, long long, int, int, cudaStream_t);            \
    int batch_stream_outc_##n(int, bool);
RDC_DECL_BATCH(f32)
RDC_DECL_BATCH(f64)
RDC_DECL_BATCH(bf16)
RDC_DECL_BATCH(f16)
#undef RDC_DECL_BATCH

cudaError_t launch_batch_step1(int prec, const GridDesc* d, const TileMap* map, int rows,
                               unsigned* q, int j, long long sbase, int sr, int ctas,
                               cudaStream_t st)
{
    switch (prec) {
        case P_F32: return launch_batch_step1_f32(d, map, rows, q, j, sbase, sr, ctas, st);
        case P_F64: return launch_batch_step1_f64(d, map, rows, q, j, sbase, sr, ctas, st);
        case P_BF16: return launch_batch_step1_bf16(d, map, rows, q, j, sbase, sr, ctas, st);
        case P_F16: return launch_batch_step1_f16(d, map, rows, q, j, sbase, sr, ctas, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_stream(int prec, const GridDesc* d, const TileMap* map, int rows,
                                unsigned* q, int k, int j, long long sbase, int sr, int ctas,
                                cudaStream_t st)
{
    switch (prec) {
        case P_F32: return launch_batch_stream_f32(d, map, rows, q, k, j, sbase, sr, ctas, st);
        case P_F64: return launch_batch_stream_f64(d, map, rows, q, k, j, sbase, sr, ctas, st);
        case P_BF16:
            return launch_batch_stream_bf16(d, map, rows, q, k, j, sbase, sr, ctas, st);
        case P_F16: return launch_batch_stream_f16(d, map, rows, q, k, j, sbase, sr, ctas, st);
    }
    return cudaErrorInvalidValue;
}

int batch_step1_cols(int prec) { return 32 * vec_cells(prec); }

int batch_stream_outc(int prec, int k, bool sr)
{
    switch (prec) {
        case P_F32: return batch_stream_outc_f32(k, sr);
        case P_F64: return batch_stream_outc_f64(k, sr);
        case P_BF16: return batch_stream_outc_bf16(k, sr);
        case P_F16: return batch_stream_outc_f16(k, sr);
    }
    return 0;
}

cudaError_t launch_step1(int prec, int mode, const Planes& g, const ModelD& m,
                         Shape1 s, cudaStream_t st)
{
    switch (prec) {
        case P_F32: return launch_step1_f32(mode, g, m, s, st);
        case P_F64: return launch_step1_f64(mode, g, m, s, st);
        case P_BF16: return launch_step1_bf16(mode, g, m, s, st);
        case P_F16: return launch_step1_f16(mode, g, m, s, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_stepk(int prec, int mode, const Planes& g, const ModelD& m,
                         ShapeK s, cudaStream_t st)
{
    switch (prec) {
        case P_F32: return launch_stepk_f32(mode, g, m, s, st);
        case P_F64: return launch_stepk_f64(mode, g, m, s, st);
        case P_BF16: return launch_stepk_bf16(mode, g, m, s, st);
        case P_F16: return launch_stepk_f16(mode, g, m, s, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_stream(int prec, const Planes& g, const ModelD& m, int k, int rows,
                          cudaStream_t st)
{
    switch (prec) {
        case P_F32: return launch_stream_f32(g, m, k, rows, st);
        case P_F64: return launch_stream_f64(g, m, k, rows, st);
        case P_BF16: return launch_stream_bf16(g, m, k, rows, st);
        case P_F16: return launch_stream_f16(g, m, k, rows, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_kblock(int prec, int mode, const Planes& g, const ModelD& m, ShapeK s,
                          cudaStream_t st)
{
    if (s.variant == 0 && mode == MODE_FULL) return launch_stream(prec, g, m, s.k, s.krows, st);
    return launch_stepk(prec, mode, g, m, s, st);
}

size_t stepk_smem_bytes(int prec, ShapeK s)
{
    switch (prec) {
        case P_F32: return stepk_smem_f32(s);
        case P_F64: return stepk_smem_f64(s);
        case P_BF16: return stepk_smem_bf16(s);
        case P_F16: return stepk_smem_f16(s);
    }
    return 0;
}
}  // namespace rdc

using namespace rdc;

// Table 1 of the paper.
static const double kEps = 0.0243, kF = 1.4, kQ = 0.002, kDu = 0.45,
                    kDt = 0.001, kDx = 0.25, kPhiActive = 0.054;

static const int kProbeChunk = 256;
static const size_t kMiscBytes = 256 + kProbeChunk * 16;

struct rdc_sim {
    int W = 0, H = 0;
    rdc_params p{};
    int prec = 0, mode = 0;
    int64_t pitch = 0;  // elements, all planes
    void* base = nullptr;
    bool owns = false;
    void* u[2] = {nullptr, nullptr};
    void* v[2] = {nullptr, nullptr};
    void* phi = nullptr;
    int cur = 0;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    unsigned char* misc = nullptr;  // flag at +0, probe cells at +256, out after
    bool owns_misc = false;
    void* stage = nullptr;
    size_t stage_bytes = 0;
    float* timelapse = nullptr;   // running maximum of u (lazily allocated)
    bool timelapse_set = false;
    int64_t steps_done = 0, launches = 0;
    double phi_max = 0.0;   // largest phi of the map (an upper bound after drawing)
    double rho = 0.0;       // stability of forward Euler at the rest state of phi_max
    bool unstable = false;  // rho > 1
    Shape1 shape1{128, 16};
    ShapeK shapek{64, 32, 1, 256};
};

static thread_local char g_err[512] = "";

int host_cuda_fail(cudaError_t e, const char* what)
{
    std::snprintf(g_err, sizeof g_err, "%s: %s (%s)", what, cudaGetErrorName(e),
                  cudaGetErrorString(e));
    // A failed runtime call leaves its (non-sticky) error as the "last error";
    // clear it so that the next kernel launch does not report it as its own.
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? RDC_ENOMEM : RDC_ECUDA;
}

#define CK(call, what)                               \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return host_cuda_fail(e_, what); \
    } while (0)

static ModelD model_of(const rdc_params& p)
{
    ModelD m;
    m.eps = p.eps;
    m.f = p.f;
    m.q = p.q;
    m.Du = p.Du;
    m.dt = p.dt;
    m.inv_dx2 = 1.0 / (p.dx * p.dx);
    m.sr = (p.flags & RDC_STOCH_ROUND) ? 1 : 0;
    m.seed = (unsigned)p.round_seed;
    return m;
}

bool host_params_valid(const rdc_params* p)
{
    if (!p) return false;
    const double vals[6] = {p->eps, p->f, p->q, p->Du, p->dt, p->dx};
    for (double x : vals)
        if (!std::isfinite(x)) return false;
    if (!(p->eps > 0.0) || !(p->q > 0.0) || !(p->q < 1.0) || !(p->dt > 0.0) ||
        !(p->dx > 0.0) || p->Du < 0.0)
        return false;
    if (!(p->f + p->q > 1.0)) return false;
    if (p->Du * p->dt / (p->dx * p->dx) > 0.25) return false;
    if (p->precision < 0 || p->precision > 3) return false;
    if (p->flags & ~(RDC_DIFFUSION_ONLY | RDC_REACTION_ONLY | RDC_STOCH_ROUND)) return false;
    if ((p->flags & RDC_DIFFUSION_ONLY) && (p->flags & RDC_REACTION_ONLY)) return false;
    const bool sr = (p->flags & RDC_STOCH_ROUND) != 0;
    if (sr && p->precision != RDC_F32_BF16STORE && p->precision != RDC_F32_F16STORE)
        return false;
    if (!sr && p->round_seed != 0) return false;
    if (p->k_block < 0 || p->k_block > 8) return false;
    return true;
}

bool host_phi_ok(double phi, const rdc_params* p)
{
    return std::isfinite(phi) && phi > p->q * (1.0 + p->f);
}

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int host_check_device()
{
    int dev = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    int major = 0, minor = 0;
    CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev), "cudaDeviceGetAttribute");
    CK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev), "cudaDeviceGetAttribute");
    if (major != 10 || minor != 3) {
        std::snprintf(g_err, sizeof g_err,
                      "librdc is built for sm_103a only; device %d is sm_%d%d",
                      dev, major, minor);
        return RDC_EUNSUPPORTED;
    }
    return RDC_OK;
}

static void default_shapes(rdc_sim* s)
{
    const int vec = vec_cells(s->prec);
    const int64_t vecs = (s->W + vec - 1) / vec;
    int bx = 128;
    if (vecs < bx) bx = (int)std::max<int64_t>(32, round_up(vecs, 32));
    const int64_t ncb = (vecs + bx - 1) / bx;
    int rows = 8;
    while (rows > 1 && ncb * ((s->H + rows - 1) / rows) < 152 * 8) rows /= 2;
    s->shape1 = Shape1{bx, rows};
    if (s->prec == P_F64)
        s->shapek = ShapeK{32, 32, 1, 256};
    else
        s->shapek = ShapeK{64, 32, 1, 256};
    // k_block = 0: temporal blocking for grids of a million cells or more in
    // the FP32-compute modes, where HBM would otherwise bound a single step
    // (measured best at 8192^2: 4 steps per launch); FP64 is bound by its
    // arithmetic, so one step per launch.  rdc_tune measures instead of
    // guessing.
    int kdef = 1;
    if (s->p.k_block == 0 && s->prec != P_F64 && s->mode == MODE_FULL &&
        (int64_t)s->W * s->H >= (1 << 20))
        kdef = 4;
    s->shapek.k = s->p.k_block == 0 ? kdef : s->p.k_block;
    s->shapek.variant = 0;
    // rows per CTA of the streamed kernel: long enough that the 2k rows of
    // overlap cost little (measured best: 64 for k <= 4, 128 beyond, on large
    // grids), shorter on small grids so that every SM gets warps
    int krows = s->shapek.k >= 5 ? 128 : 64;
    while (krows > 16 && (int64_t)((s->W + 111) / 112) * ((s->H + krows - 1) / krows) < 152 * 16)
        krows /= 2;
    // and few enough CTA rows for the 65535 limit of gridDim.y on tall grids
    while ((s->H + krows - 1) / krows > 65535) krows *= 2;
    s->shapek.krows = krows;
}

static void destroy_impl(rdc_sim* s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->owns && s->base) cudaFree(s->base);
    if (s->owns_misc && s->misc) cudaFree(s->misc);
    if (s->stage) cudaFree(s->stage);
    if (s->timelapse) cudaFree(s->timelapse);
    if (s->owns_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

static int ensure_stage(rdc_sim* s, size_t bytes)
{
    if (s->stage_bytes >= bytes) return RDC_OK;
    if (s->stage) {
        CK(cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
        cudaFree(s->stage);
        s->stage = nullptr;
        s->stage_bytes = 0;
    }
    CK(cudaMalloc(&s->stage, bytes), "cudaMalloc(stage)");
    s->stage_bytes = bytes;
    return RDC_OK;
}

// Host phi (float or double, packed) -> device phi plane.
static int upload_phi(rdc_sim* s, const void* phi_host, int dtype)
{
    const int pb = phi_bytes(s->prec);
    const bool direct = (dtype == 0 && pb == 4) || (dtype == 1 && pb == 8);
    if (direct) {
        CK(cudaMemcpy2DAsync(s->phi, (size_t)s->pitch * pb, phi_host, (size_t)s->W * pb,
                             (size_t)s->W * pb, s->H, cudaMemcpyHostToDevice, s->stream),
           "cudaMemcpy2DAsync(phi)");
        return RDC_OK;
    }
    const size_t bytes = (size_t)s->W * s->H * dtype_bytes(dtype);
    int rc = ensure_stage(s, bytes);
    if (rc) return rc;
    CK(cudaMemcpyAsync(s->stage, phi_host, bytes, cudaMemcpyHostToDevice, s->stream),
       "cudaMemcpyAsync(phi)");
    CK(launch_phi_in(s->prec, dtype, s->stage, s->phi, s->W, s->H, s->pitch, s->stream),
       "phi conversion kernel");
    return RDC_OK;
}

// Smallest and largest value of x[k0, k1) and whether any is a NaN, over
// eight independent lanes without branches (so the compiler can keep the
// lanes in vector registers).
template <typename T>
static void minmax_range(const T* x, int64_t k0, int64_t k1, double* lo, double* hi, bool* nan)
{
    T mn[8], mx[8];
    unsigned bad = 0;
    for (int i = 0; i < 8; ++i) {
        mn[i] = std::numeric_limits<T>::infinity();
        mx[i] = -std::numeric_limits<T>::infinity();
    }
    int64_t k = k0;
    for (; k + 8 <= k1; k += 8)
        for (int i = 0; i < 8; ++i) {
            const T v = x[k + i];
            mn[i] = v < mn[i] ? v : mn[i];
            mx[i] = v > mx[i] ? v : mx[i];
            bad |= (unsigned)(v != v);
        }
    for (; k < k1; ++k) {
        const T v = x[k];
        mn[0] = v < mn[0] ? v : mn[0];
        mx[0] = v > mx[0] ? v : mx[0];
        bad |= (unsigned)(v != v);
    }
    T a = mn[0], b = mx[0];
    for (int i = 1; i < 8; ++i) {
        a = mn[i] < a ? mn[i] : a;
        b = mx[i] > b ? mx[i] : b;
    }
    *lo = (double)a;
    *hi = (double)b;
    *nan = bad != 0;
}

// Validates every phi value and finds the largest: the map is valid when no
// value is a NaN and its smallest and largest values pass host_phi_ok (every
// value between them then does).  Maps of more than 2^20 values are split
// over host threads.
bool host_scan_phi(const void* phi_host, int dtype, int64_t n, const rdc_params* p,
                   double* mx)
{
    auto scan = [&](int64_t k0, int64_t k1, double* lo, double* hi, bool* nan) {
        if (dtype == 0) minmax_range((const float*)phi_host, k0, k1, lo, hi, nan);
        else minmax_range((const double*)phi_host, k0, k1, lo, hi, nan);
    };
    const int64_t kChunk = int64_t(1) << 20;
    unsigned hw = std::thread::hardware_concurrency();
    const int nt = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<unsigned>(hw ? hw : 1, 16u), (n + kChunk - 1) / kChunk));
    std::vector<double> lo(nt, INFINITY), hi(nt, -INFINITY);
    std::vector<char> nan(nt, 0);
    const int64_t per = (n + nt - 1) / nt;
    auto part = [&](int t) {
        const int64_t k0 = std::min(n, t * per), k1 = std::min(n, k0 + per);
        bool b = false;
        if (k1 > k0) scan(k0, k1, &lo[t], &hi[t], &b);
        nan[t] = b ? 1 : 0;
    };
    if (nt == 1) {
        part(0);
    } else {
        std::vector<std::thread> th;
        for (int t = 1; t < nt; ++t) th.emplace_back(part, t);
        part(0);
        for (auto& x : th) x.join();
    }
    double a = INFINITY, b = -INFINITY;
    for (int t = 0; t < nt; ++t) {
        if (nan[t]) return false;
        a = std::min(a, lo[t]);
        b = std::max(b, hi[t]);
    }
    if (n > 0 && !(host_phi_ok(a, p) && host_phi_ok(b, p))) return false;
    *mx = b;
    return true;
}

// Records rho and the unstable flag of the current phi_max.
static void update_stability(rdc_sim* s)
{
    double rho = std::nan("");
    const int rc = host_stability(s->p, s->phi_max, &rho);
    s->rho = rho;
    s->unstable = rc != RDC_OK;  // unstable, or (caller-owned map) no rest state at all
}

static int create_common(rdc_grid g, const rdc_params* p, const void* phi_host,
                         int phi_dtype, void* stream, void* const* ext_u,
                         void* const* ext_v, const void* ext_phi,
                         size_t ext_pitch_bytes, rdc_sim** out)
{
    NvtxRange nvtx("rdc_create");
    if (!out) return RDC_EINVAL;
    *out = nullptr;
    if (g.width < 1 || g.height < 1 || !host_params_valid(p)) return RDC_EINVAL;
    const int64_t n = (int64_t)g.width * g.height;
    double phi_max = kPhiActive;
    if (phi_host) {
        if (!host_scan_phi(phi_host, phi_dtype, n, p, &phi_max)) return RDC_EINVAL;
    } else if (!ext_u && !host_phi_ok(kPhiActive, p)) {
        return RDC_EINVAL;
    }
    const int prec = p->precision;
    const int esz = state_bytes(prec);
    if (ext_u) {
        for (int b = 0; b < 2; ++b)
            if (!ext_u[b] || !ext_v[b] || ((uintptr_t)ext_u[b] % 16) || ((uintptr_t)ext_v[b] % 16))
                return RDC_EINVAL;
        if (!ext_phi || ((uintptr_t)ext_phi % 16)) return RDC_EINVAL;
        if (ext_pitch_bytes % 16 || ext_pitch_bytes < (size_t)g.width * esz ||
            ext_pitch_bytes % esz)
            return RDC_EINVAL;
    }
    int rc = host_check_device();
    if (rc) return rc;

    rdc_sim* s = new (std::nothrow) rdc_sim();
    if (!s) return RDC_ENOMEM;
    s->W = g.width;
    s->H = g.height;
    s->p = *p;
    s->prec = prec;
    s->mode = p->flags & (RDC_DIFFUSION_ONLY | RDC_REACTION_ONLY);
    s->phi_max = phi_max;
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete s;
            return host_cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        s->owns_stream = true;
    }

    if (ext_u) {
        s->pitch = (int64_t)(ext_pitch_bytes / esz);
        s->u[0] = ext_u[0];
        s->u[1] = ext_u[1];
        s->v[0] = ext_v[0];
        s->v[1] = ext_v[1];
        s->phi = const_cast<void*>(ext_phi);
        cudaError_t e = cudaMalloc((void**)&s->misc, kMiscBytes);
        if (e != cudaSuccess) {
            destroy_impl(s);
            return host_cuda_fail(e, "cudaMalloc(scratch)");
        }
        s->owns_misc = true;
        // The caller's phi map is not read on the host: its largest value
        // (for the stability check) comes from the device.
        long long mx = LLONG_MIN;
        long long* dmx = reinterpret_cast<long long*>(s->misc);
        e = cudaMemcpyAsync(dmx, &mx, sizeof mx, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess)
            e = launch_phi_max(prec, s->phi, s->W, s->H, s->pitch, dmx, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&mx, dmx, sizeof mx, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) {
            destroy_impl(s);
            return host_cuda_fail(e, "phi maximum");
        }
        const long long bits = mx >= 0 ? mx : (mx ^ 0x7FFFFFFFFFFFFFFFLL);
        std::memcpy(&s->phi_max, &bits, sizeof bits);
    } else {
        s->pitch = round_up(g.width, 64);
        const size_t sp = (size_t)round_up((int64_t)s->pitch * s->H * esz, 256);
        const size_t pp = (size_t)round_up((int64_t)s->pitch * s->H * phi_bytes(prec), 256);
        const size_t total = 4 * sp + pp + kMiscBytes;
        cudaError_t e = cudaMalloc(&s->base, total);
        if (e != cudaSuccess) {
            destroy_impl(s);
            return host_cuda_fail(e, "cudaMalloc(planes)");
        }
        s->owns = true;
        unsigned char* b = (unsigned char*)s->base;
        s->u[0] = b;
        s->u[1] = b + sp;
        s->v[0] = b + 2 * sp;
        s->v[1] = b + 3 * sp;
        s->phi = b + 4 * sp;
        s->misc = b + 4 * sp + pp;
        e = cudaMemsetAsync(s->base, 0, total, s->stream);
        if (e != cudaSuccess) {
            destroy_impl(s);
            return host_cuda_fail(e, "cudaMemsetAsync");
        }
        if (phi_host) {
            rc = upload_phi(s, phi_host, phi_dtype);
        } else {
            e = launch_fill_phi(prec, s->phi, s->W, s->H, s->pitch, kPhiActive, s->stream);
            rc = e == cudaSuccess ? RDC_OK : host_cuda_fail(e, "phi fill kernel");
        }
        if (rc == RDC_OK) {
            e = launch_rest(prec, s->u[0], s->v[0], s->phi, s->W, s->H, s->pitch, p->f,
                            p->q, s->stream);
            rc = e == cudaSuccess ? RDC_OK : host_cuda_fail(e, "rest-state kernel");
        }
        if (rc == RDC_OK) {
            e = cudaStreamSynchronize(s->stream);
            rc = e == cudaSuccess ? RDC_OK : host_cuda_fail(e, "cudaStreamSynchronize");
        }
        if (rc != RDC_OK) {
            destroy_impl(s);
            return rc;
        }
    }
    default_shapes(s);
    update_stability(s);
    *out = s;
    return RDC_OK;
}

int host_stability(const rdc_params& p, double phi_max, double* rho_out)
{
    double us = 0.0;
    if (rdc_rest_state(phi_max, p.f, p.q, &us) != RDC_OK) return RDC_EINVAL;
    // Jacobian of Eq. 1's reaction part at u = v = u*:
    //   dR/du = 1 - 2u - (f v + phi) 2q/(u+q)^2,  dR/dv = -f (u-q)/(u+q)
    const double a = 1.0 - 2.0 * us - (p.f * us + phi_max) * 2.0 * p.q / ((us + p.q) * (us + p.q));
    const double b = -p.f * (us - p.q) / (us + p.q);
    const double lap_min = -8.0 * p.Du / (p.dx * p.dx);
    double rho = 0.0;
    for (int k = 0; k <= 64; ++k) {
        const double shift = lap_min * k / 64.0;
        // J = [[a/eps + shift, b/eps], [1, -1]]
        const double j11 = a / p.eps + shift, j12 = b / p.eps, j21 = 1.0, j22 = -1.0;
        const double tr = j11 + j22, det = j11 * j22 - j12 * j21;
        const std::complex<double> disc = std::sqrt(std::complex<double>(tr * tr - 4.0 * det, 0.0));
        const std::complex<double> l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
        rho = std::max(rho, std::abs(1.0 + p.dt * l1));
        rho = std::max(rho, std::abs(1.0 + p.dt * l2));
    }
    *rho_out = rho;
    return rho > 1.0 ? RDC_EUNSTABLE_WARN : RDC_OK;
}

extern "C" {

int rdc_params_default(rdc_params* out)
{
    if (!out) return RDC_EINVAL;
    std::memset(out, 0, sizeof *out);
    out->eps = kEps;
    out->f = kF;
    out->q = kQ;
    out->Du = kDu;
    out->dt = kDt;
    out->dx = kDx;
    out->precision = RDC_F32;
    out->flags = 0;
    out->k_block = 0;
    out->round_seed = 0;
    return RDC_OK;
}

int rdc_create(rdc_grid g, const rdc_params* p, const float* phi_host,
               void* stream, rdc_sim** out)
{
    return create_common(g, p, phi_host, 0, stream, nullptr, nullptr, nullptr, 0, out);
}

int rdc_create_f64phi(rdc_grid g, const rdc_params* p, const double* phi_host,
                      void* stream, rdc_sim** out)
{
    return create_common(g, p, phi_host, 1, stream, nullptr, nullptr, nullptr, 0, out);
}

int rdc_create_ext(rdc_grid g, const rdc_params* p, void* const dev_u[2],
                   void* const dev_v[2], const void* dev_phi, size_t pitch_bytes,
                   void* stream, rdc_sim** out)
{
    if (!dev_u || !dev_v) return RDC_EINVAL;
    return create_common(g, p, nullptr, 0, stream, dev_u, dev_v, dev_phi, pitch_bytes, out);
}

void rdc_destroy(rdc_sim* sim) { destroy_impl(sim); }

int rdc_reset_rest(rdc_sim* s)
{
    if (!s) return RDC_EINVAL;
    CK(launch_rest(s->prec, s->u[0], s->v[0], s->phi, s->W, s->H, s->pitch, s->p.f,
                   s->p.q, s->stream),
       "rest-state kernel");
    s->cur = 0;
    s->steps_done = 0;
    return RDC_OK;
}

int rdc_set_step_index(rdc_sim* s, int64_t n)
{
    if (!s || n < 0) return RDC_EINVAL;
    s->steps_done = n;
    return RDC_OK;
}

int rdc_set_phi(rdc_sim* s, const void* phi_host, int32_t dtype)
{
    if (!s || !phi_host || (dtype != 0 && dtype != 1)) return RDC_EINVAL;
    double mx = 0.0;
    if (!host_scan_phi(phi_host, dtype, (int64_t)s->W * s->H, &s->p, &mx)) return RDC_EINVAL;
    int rc = upload_phi(s, phi_host, dtype);
    if (rc) return rc;
    s->phi_max = mx;
    update_stability(s);
    return rdc_reset_rest(s);
}

int rdc_seed(rdc_sim* s, double cx, double cy, double r, double value)
{
    if (!s || !std::isfinite(cx) || !std::isfinite(cy) || !std::isfinite(value) ||
        !(r >= 0.0) || !(r < 16777216.0))
        return RDC_EINVAL;
    CK(launch_seed(s->prec, s->u[s->cur], s->W, s->H, s->pitch, cx, cy, r, value, s->stream),
       "seed kernel");
    return RDC_OK;
}

int rdc_set_state(rdc_sim* s, const void* u_host, const void* v_host, int32_t dtype)
{
    if (!s || dtype < 0 || dtype > 3) return RDC_EINVAL;
    const int esz = state_bytes(s->prec);
    const void* src[2] = {u_host, v_host};
    void* dst[2] = {s->u[s->cur], s->v[s->cur]};
    for (int b = 0; b < 2; ++b) {
        if (!src[b]) continue;
        if (dtype == s->prec) {
            CK(cudaMemcpy2DAsync(dst[b], (size_t)s->pitch * esz, src[b], (size_t)s->W * esz,
                                 (size_t)s->W * esz, s->H, cudaMemcpyHostToDevice, s->stream),
               "cudaMemcpy2DAsync(state)");
        } else {
            const size_t bytes = (size_t)s->W * s->H * dtype_bytes(dtype);
            int rc = ensure_stage(s, bytes);
            if (rc) return rc;
            CK(cudaMemcpyAsync(s->stage, src[b], bytes, cudaMemcpyHostToDevice, s->stream),
               "cudaMemcpyAsync(state)");
            CK(launch_pack_in(s->prec, dtype, s->stage, dst[b], s->W, s->H, s->pitch, s->stream),
               "state conversion kernel");
        }
    }
    return RDC_OK;
}

int rdc_step(rdc_sim* s, int64_t n)
{
    NvtxRange nvtx("rdc_step");
    if (!s || n < 0) return RDC_EINVAL;
    ModelD m = model_of(s->p);
    int64_t left = n;
    const int k = s->shapek.k;
    while (left > 0) {
        Planes g{s->u[s->cur], s->v[s->cur], s->phi, s->u[1 - s->cur], s->v[1 - s->cur],
                 s->W, s->H, s->pitch};
        cudaError_t e;
        int done;
        m.step0 = s->steps_done;  // index of the state this launch reads
        m.flip = (int)(s->launches & 1);  // alternate the single step's sweep direction
        if (k > 1 && left >= k) {
            e = launch_kblock(s->prec, s->mode, g, m, s->shapek, s->stream);
            done = k;
        } else {
            e = launch_step1(s->prec, s->mode, g, m, s->shape1, s->stream);
            done = 1;
        }
        if (e != cudaSuccess) return host_cuda_fail(e, "step kernel");
        s->cur = 1 - s->cur;
        s->steps_done += done;
        s->launches += 1;
        left -= done;
    }
    return RDC_OK;
}

int rdc_check(rdc_sim* s, int64_t* first_bad)
{
    if (!s) return RDC_EINVAL;
    unsigned long long* flag = (unsigned long long*)s->misc;
    CK(cudaMemsetAsync(flag, 0xFF, sizeof(unsigned long long), s->stream), "cudaMemsetAsync(flag)");
    CK(launch_health(s->prec, s->u[s->cur], s->W, s->H, s->pitch, s->p.q, flag, s->stream),
       "health kernel");
    unsigned long long h = 0;
    CK(cudaMemcpyAsync(&h, flag, sizeof h, cudaMemcpyDeviceToHost, s->stream), "cudaMemcpyAsync(flag)");
    CK(cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    const bool bad = (h != ~0ull);
    if (first_bad) *first_bad = bad ? (int64_t)h : -1;
    return bad ? RDC_ENONFINITE : RDC_OK;
}

int rdc_read(rdc_sim* s, void* u_out, void* v_out, int32_t dtype)
{
    NvtxRange nvtx("rdc_read");
    if (!s || dtype < 0 || dtype > 3) return RDC_EINVAL;
    const int esz = state_bytes(s->prec);
    const void* src[2] = {s->u[s->cur], s->v[s->cur]};
    void* dst[2] = {u_out, v_out};
    for (int b = 0; b < 2; ++b) {
        if (!dst[b]) continue;
        if (dtype == s->prec) {
            CK(cudaMemcpy2DAsync(dst[b], (size_t)s->W * esz, src[b], (size_t)s->pitch * esz,
                                 (size_t)s->W * esz, s->H, cudaMemcpyDeviceToHost, s->stream),
               "cudaMemcpy2DAsync(read)");
        } else {
            const size_t bytes = (size_t)s->W * s->H * dtype_bytes(dtype);
            int rc = ensure_stage(s, bytes);
            if (rc) return rc;
            CK(launch_pack_out(s->prec, dtype, src[b], s->stage, s->W, s->H, s->pitch, s->stream),
               "state conversion kernel");
            CK(cudaMemcpyAsync(dst[b], s->stage, bytes, cudaMemcpyDeviceToHost, s->stream),
               "cudaMemcpyAsync(read)");
            CK(cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
        }
    }
    return rdc_check(s, nullptr);
}

// Copies rows of the current u and v planes to (get) or from (put) caller
// buffers of the storage type, one 2-D copy per plane on the sim's stream.
static int copy_rows(rdc_sim* s, int32_t row0, int32_t nrows, void* const bufs[2],
                     size_t pitch_bytes, bool get)
{
    if (!s || row0 < 0 || nrows < 0 || (int64_t)row0 + nrows > s->H) return RDC_EINVAL;
    const size_t esz = (size_t)state_bytes(s->prec);
    const size_t row_bytes = (size_t)s->W * esz;
    if (pitch_bytes == 0) pitch_bytes = row_bytes;
    if (pitch_bytes < row_bytes) return RDC_EINVAL;
    if (nrows == 0) return RDC_OK;
    void* planes[2] = {s->u[s->cur], s->v[s->cur]};
    const size_t plane_pitch = (size_t)s->pitch * esz;
    for (int b = 0; b < 2; ++b) {
        if (!bufs[b]) continue;
        char* rows = (char*)planes[b] + (size_t)row0 * plane_pitch;
        if (get)
            CK(cudaMemcpy2DAsync(bufs[b], pitch_bytes, rows, plane_pitch, row_bytes, nrows,
                                 cudaMemcpyDefault, s->stream),
               "cudaMemcpy2DAsync(get rows)");
        else
            CK(cudaMemcpy2DAsync(rows, plane_pitch, bufs[b], pitch_bytes, row_bytes, nrows,
                                 cudaMemcpyDefault, s->stream),
               "cudaMemcpy2DAsync(put rows)");
    }
    return RDC_OK;
}

int rdc_get_rows(rdc_sim* s, int32_t row0, int32_t nrows, void* u_dst, void* v_dst,
                 size_t pitch_bytes)
{
    void* bufs[2] = {u_dst, v_dst};
    return copy_rows(s, row0, nrows, bufs, pitch_bytes, true);
}

int rdc_put_rows(rdc_sim* s, int32_t row0, int32_t nrows, const void* u_src,
                 const void* v_src, size_t pitch_bytes)
{
    void* bufs[2] = {const_cast<void*>(u_src), const_cast<void*>(v_src)};
    return copy_rows(s, row0, nrows, bufs, pitch_bytes, false);
}

int rdc_probe(rdc_sim* s, int32_t n, const int64_t* cells, double* out)
{
    if (!s || n < 0 || (n > 0 && (!cells || !out))) return RDC_EINVAL;
    const int64_t ncell = (int64_t)s->W * s->H;
    for (int32_t k = 0; k < n; ++k)
        if (cells[k] < 0 || cells[k] >= ncell) return RDC_EINVAL;
    int64_t* d_cells = (int64_t*)(s->misc + 256);
    double* d_out = (double*)(s->misc + 256 + kProbeChunk * 8);
    for (int32_t k0 = 0; k0 < n; k0 += kProbeChunk) {
        const int m = std::min<int32_t>(kProbeChunk, n - k0);
        CK(cudaMemcpyAsync(d_cells, cells + k0, m * sizeof(int64_t), cudaMemcpyHostToDevice,
                           s->stream),
           "cudaMemcpyAsync(probe)");
        CK(launch_probe(s->prec, s->u[s->cur], s->W, s->pitch, d_cells, m, d_out, s->stream),
           "probe kernel");
        CK(cudaMemcpyAsync(out + k0, d_out, m * sizeof(double), cudaMemcpyDeviceToHost, s->stream),
           "cudaMemcpyAsync(probe)");
        CK(cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    }
    return RDC_OK;
}

int rdc_snap_segment(double x0, double y0, double x1, double y1, double snap_deg,
                     double* x1s, double* y1s)
{
    if (!x1s || !y1s || !std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(x1) ||
        !std::isfinite(y1) || !(snap_deg > 0.0) || !std::isfinite(snap_deg))
        return RDC_EINVAL;
    // The documented sequence; host code is compiled without contraction.
    const double dx = x1 - x0, dy = y1 - y0;
    const double len = std::hypot(dx, dy);
    double a = std::atan2(dy, dx) * (180.0 / 3.14159265358979323846);
    a = std::round(a / snap_deg) * snap_deg;
    const double r = a * (3.14159265358979323846 / 180.0);
    *x1s = x0 + len * std::cos(r);
    *y1s = y0 + len * std::sin(r);
    return RDC_OK;
}

int rdc_draw_line(rdc_sim* s, double x0, double y0, double x1, double y1, double width,
                  double value, double snap_deg)
{
    if (!s || !std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(x1) ||
        !std::isfinite(y1) || !(width >= 0.0) || !(width < 1e7) || !host_phi_ok(value, &s->p) ||
        !(snap_deg >= 0.0) || !std::isfinite(snap_deg))
        return RDC_EINVAL;
    if (snap_deg > 0.0) {
        int rc = rdc_snap_segment(x0, y0, x1, y1, snap_deg, &x1, &y1);
        if (rc) return rc;
    }
    CK(launch_draw_line(s->prec, s->phi, s->W, s->H, s->pitch, x0, y0, x1, y1, width, value,
                        s->stream),
       "draw kernel");
    if (value > s->phi_max) s->phi_max = value;
    update_stability(s);
    return RDC_OK;
}

int rdc_read_phi(rdc_sim* s, void* out, int32_t dtype)
{
    if (!s || !out || (dtype != RDC_DTYPE_F32 && dtype != RDC_DTYPE_F64)) return RDC_EINVAL;
    const int pb = phi_bytes(s->prec);
    const bool direct = (dtype == RDC_DTYPE_F32 && pb == 4) || (dtype == RDC_DTYPE_F64 && pb == 8);
    if (direct) {
        CK(cudaMemcpy2DAsync(out, (size_t)s->W * pb, s->phi, (size_t)s->pitch * pb,
                             (size_t)s->W * pb, s->H, cudaMemcpyDeviceToHost, s->stream),
           "cudaMemcpy2DAsync(phi)");
    } else {
        const size_t bytes = (size_t)s->W * s->H * dtype_bytes(dtype);
        int rc = ensure_stage(s, bytes);
        if (rc) return rc;
        // phi planes are float or double: the state conversion kernels apply
        CK(launch_pack_out(pb == 8 ? P_F64 : P_F32, dtype, s->phi, s->stage, s->W, s->H,
                           s->pitch, s->stream),
           "phi conversion kernel");
        CK(cudaMemcpyAsync(out, s->stage, bytes, cudaMemcpyDeviceToHost, s->stream),
           "cudaMemcpyAsync(phi)");
    }
    CK(cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    return RDC_OK;
}

int rdc_fill_phi(rdc_sim* s, double value)
{
    if (!s || !host_phi_ok(value, &s->p)) return RDC_EINVAL;
    CK(launch_fill_phi(s->prec, s->phi, s->W, s->H, s->pitch, value, s->stream), "fill kernel");
    s->phi_max = value;
    update_stability(s);
    return RDC_OK;
}

int rdc_timelapse_record(rdc_sim* s, int32_t reset)
{
    if (!s || reset < 0 || reset > 1) return RDC_EINVAL;
    if (!s->timelapse) {
        CK(cudaMalloc((void**)&s->timelapse, (size_t)s->pitch * s->H * sizeof(float)),
           "cudaMalloc(timelapse)");
        reset = 1;
    }
    if (!s->timelapse_set) reset = 1;
    CK(launch_timelapse(s->prec, s->u[s->cur], s->timelapse, s->W, s->H, s->pitch, s->pitch,
                        reset, s->stream),
       "timelapse kernel");
    s->timelapse_set = true;
    return RDC_OK;
}

int rdc_render(rdc_sim* s, int32_t what, float u_scale, float v_scale, double phi_threshold,
               void* rgba, int32_t out_on_device)
{
    if (!s || !rgba || (what != 0 && what != 1) || !std::isfinite(u_scale) ||
        !std::isfinite(v_scale) || std::isnan(phi_threshold) ||
        (out_on_device != 0 && out_on_device != 1))
        return RDC_EINVAL;
    if (what == 1 && !s->timelapse_set) return RDC_EINVAL;
    const size_t bytes = (size_t)s->W * s->H * 4;
    void* dst = rgba;
    if (!out_on_device) {
        int rc = ensure_stage(s, bytes);
        if (rc) return rc;
        dst = s->stage;
    } else if ((uintptr_t)rgba % 4) {
        return RDC_EINVAL;
    }
    CK(launch_render(s->prec, s->u[s->cur], s->v[s->cur], s->phi,
                     what == 1 ? s->timelapse : nullptr, s->W, s->H, s->pitch, s->pitch, u_scale,
                     v_scale, phi_threshold, dst, s->stream),
       "render kernel");
    if (!out_on_device) {
        CK(cudaMemcpyAsync(rgba, dst, bytes, cudaMemcpyDeviceToHost, s->stream),
           "cudaMemcpyAsync(render)");
        CK(cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    }
    return RDC_OK;
}

int rdc_sync(rdc_sim* s)
{
    if (!s) return RDC_EINVAL;
    CK(cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    return RDC_OK;
}

int rdc_rest_state(double phi, double f, double q, double* u_star)
{
    if (!u_star || !(q > 0.0 && q < 1.0) || !(f + q > 1.0) || !std::isfinite(f) ||
        !(phi > q * (1.0 + f)) || !std::isfinite(phi))
        return RDC_EINVAL;
    // Same rule as the device initialiser.  This translation unit's host code
    // is compiled with -ffp-contract=off, so each operation rounds once.
    const double a2 = (f + q) - 1.0;
    const double a1 = (phi - q) - f * q;
    const double a0 = -(phi * q);
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 2000; ++it) {
        const double mid = lo + (hi - lo) * 0.5;
        if (mid == lo || mid == hi) break;
        const double pv = ((mid + a2) * mid + a1) * mid + a0;
        if (pv < 0.0) lo = mid; else hi = mid;
    }
    *u_star = hi;
    return RDC_OK;
}

int rdc_stability(rdc_sim* s, double* rho_out)
{
    if (!s || !rho_out) return RDC_EINVAL;
    return host_stability(s->p, s->phi_max, rho_out);
}

int rdc_get_view(rdc_sim* s, rdc_view* out)
{
    if (!s || !out) return RDC_EINVAL;
    out->u = s->u[s->cur];
    out->v = s->v[s->cur];
    out->phi = s->phi;
    out->pitch_bytes = (size_t)s->pitch * state_bytes(s->prec);
    out->phi_pitch_bytes = (size_t)s->pitch * phi_bytes(s->prec);
    out->width = s->W;
    out->height = s->H;
    out->precision = s->prec;
    out->elem_bytes = state_bytes(s->prec);
    out->steps_done = s->steps_done;
    out->launches = s->launches;
    out->stream = (void*)s->stream;
    out->unstable = s->unstable ? 1 : 0;
    out->reserved = 0;
    out->stability_rho = s->rho;
    return RDC_OK;
}

int rdc_get_shape(rdc_sim* s, rdc_launch_shape* out)
{
    if (!s || !out) return RDC_EINVAL;
    out->bx = s->shape1.bx;
    out->rows = s->shape1.rows;
    out->tx = s->shapek.tx;
    out->ty = s->shapek.ty;
    out->nthreads = s->shapek.nthreads;
    out->k = s->shapek.k;
    out->variant = s->shapek.variant;
    out->krows = s->shapek.krows;
    return RDC_OK;
}

int rdc_set_shape(rdc_sim* s, const rdc_launch_shape* in)
{
    if (!s || !in) return RDC_EINVAL;
    if (in->bx < 32 || in->bx > 256 || in->bx % 32 || in->rows < 1) return RDC_EINVAL;
    if (in->k < 1 || in->k > 8 || in->tx < 1 || in->ty < 1 || in->nthreads < 32 ||
        in->nthreads > 512 || in->nthreads % 32)
        return RDC_EINVAL;
    if (in->variant < 0 || in->variant > 1 || in->krows < 1) return RDC_EINVAL;
    ShapeK sk{in->tx, in->ty, in->k, in->nthreads, in->variant, in->krows};
    if (in->k > 1 && stepk_smem_bytes(s->prec, sk) > 227 * 1024) return RDC_EINVAL;
    if (in->k > 1 && (s->H + in->krows - 1) / in->krows > 65535) return RDC_EINVAL;
    if (in->k > 1 && (s->H + in->ty - 1) / in->ty > 65535) return RDC_EINVAL;
    s->shape1 = Shape1{in->bx, in->rows};
    s->shapek = sk;
    return RDC_OK;
}

int rdc_tune(rdc_sim* s, int32_t reps, rdc_launch_shape* out, double* best_gcups)
{
    NvtxRange nvtx("rdc_tune");
    if (!s || reps < 1) return RDC_EINVAL;
    const ModelD m = model_of(s->p);
    const Planes g{s->u[s->cur], s->v[s->cur], s->phi, s->u[1 - s->cur], s->v[1 - s->cur],
                   s->W, s->H, s->pitch};
    const double cells = (double)s->W * s->H;
    struct Cand {
        bool kblock;  // false: single-step kernel with s1; true: k-step kernel with sk
        Shape1 s1;
        ShapeK sk;
    };
    std::vector<Cand> cands;
    ShapeK k1 = s->shapek;
    k1.k = 1;
    for (int rows : {4, 8, 16, 32}) cands.push_back({false, Shape1{s->shape1.bx, rows}, k1});
    for (int k : {2, 3, 4, 5, 6, 7, 8}) {
        if (s->mode == MODE_FULL)  // the streamed kernel serves the full model only
            for (int krows : {32, 64, 128, 256})
                cands.push_back({true, s->shape1, ShapeK{64, 32, k, 256, 0, krows}});
        for (int ty : {32, 64})
            cands.push_back({true, s->shape1, ShapeK{64, ty, k, ty == 64 ? 512 : 256, 1, 64}});
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "cudaEventCreate");
    cudaError_t ee = cudaEventCreate(&e1);
    if (ee != cudaSuccess) {
        cudaEventDestroy(e0);
        return host_cuda_fail(ee, "cudaEventCreate");
    }
    double best = -1.0;
    Cand pick{s->shapek.k > 1, s->shape1, s->shapek};
    int rc = RDC_OK;
    for (const Cand& c : cands) {
        const bool use_k = c.kblock;
        if (use_k && c.sk.variant == 1 && stepk_smem_bytes(s->prec, c.sk) > 227 * 1024) continue;
        // shapes whose CTA rows exceed gridDim.y's 65535 on a tall grid
        if (use_k && (s->H + (c.sk.variant == 0 ? c.sk.krows : c.sk.ty) - 1) /
                             (c.sk.variant == 0 ? c.sk.krows : c.sk.ty) > 65535)
            continue;
        // each timed launch reads the current buffers and writes the spare ones
        auto launch = [&]() {
            return use_k ? launch_kblock(s->prec, s->mode, g, m, c.sk, s->stream)
                         : launch_step1(s->prec, s->mode, g, m, c.s1, s->stream);
        };
        cudaError_t e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e0, s->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = host_cuda_fail(e, "autotune launch");
            break;
        }
        const double rate = cells * (use_k ? c.sk.k : 1) * reps / (ms * 1e-3);
        if (rate > best) {
            best = rate;
            pick = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    s->shape1 = pick.s1;
    s->shapek = pick.sk;
    if (best_gcups) *best_gcups = best / 1e9;
    return out ? rdc_get_shape(s, out) : RDC_OK;
}

const char* rdc_status_str(int status)
{
    switch (status) {
        case RDC_OK: return "RDC_OK";
        case RDC_EINVAL: return "RDC_EINVAL: invalid argument";
        case RDC_ENOMEM: return "RDC_ENOMEM: allocation failed";
        case RDC_ECUDA: return "RDC_ECUDA: CUDA call failed";
        case RDC_ENONFINITE: return "RDC_ENONFINITE: non-finite u or u + q <= 0";
        case RDC_ETIMEOUT: return "RDC_ETIMEOUT: bounded device wait gave up";
        case RDC_EUNSTABLE_WARN: return "RDC_EUNSTABLE_WARN: forward Euler unstable at rest";
        case RDC_EUNSUPPORTED: return "RDC_EUNSUPPORTED: not supported by this build or device";
    }
    return "unknown rdc status";
}

const char* rdc_last_error(void) { return g_err; }

}  // extern "C"
