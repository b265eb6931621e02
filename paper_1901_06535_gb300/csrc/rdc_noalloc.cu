// rdc_step_noalloc: advance caller-owned state buffers by n Euler steps
// without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc -- applications whose
// device memory is handed out by their own pool (a framework's caching
// allocator that has reserved the device), where a library's own allocation
// could fail or fragment that pool; latency-bound loops (interactive serving)
// where cudaMalloc and cudaFree would synchronise the device and stall the
// work of every other stream; and processes that must know their device
// footprint up front.  The simulation handle API allocates its planes and a
// small scratch area; this entry point takes every input and output from the
// caller instead.
//
// The only memory it uses beyond the caller's buffers is g_scratch below: a
// file-scope device array of a fixed size that every GPU loading this
// library holds until the process exits.  It stores the intermediate state
// of multi-step calls (u and v of one ping-pong buffer) and the health flag.
// Host code never dereferences the symbol: it asks the runtime for the array's
// device address once per device (cudaGetSymbolAddress) and passes that
// address to the kernels.
#include <mutex>

#include "rdc.h"
#include "rdc_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB, shared by all calls
constexpr size_t kFlagBytes = 256;                  // health flag, then the planes

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[64] = {nullptr};   // device address of g_scratch, per device

// RDC_ECUDA, after clearing the failed call's error from the runtime's
// last-error state (so that a later launch does not report it).
int cuda_error()
{
    (void)cudaGetLastError();
    return RDC_ECUDA;
}

// Device address of g_scratch on the current device, looked up once per device
// with that device current.
int scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error();
    if (dev < 0 || dev >= 64) return RDC_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_error();
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RDC_OK;
}

bool params_ok(const rdc_params* p)
{
    if (!p) return false;
    const double v[6] = {p->eps, p->f, p->q, p->Du, p->dt, p->dx};
    for (double x : v)
        if (!(x == x) || x - x != 0.0) return false;  // NaN or infinite
    if (!(p->eps > 0.0) || !(p->q > 0.0) || !(p->q < 1.0) || !(p->dt > 0.0) ||
        !(p->dx > 0.0) || p->Du < 0.0 || !(p->f + p->q > 1.0))
        return false;
    if (p->Du * p->dt / (p->dx * p->dx) > 0.25) return false;
    if (p->precision < 0 || p->precision > 3 || p->flags < 0 || p->flags > 2) return false;
    if (p->k_block < 0 || p->k_block > 8 || p->round_seed != 0) return false;
    return true;
}

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Whether the byte ranges [a, a + na) and [b, b + nb) share a byte.
bool overlap(const void* a, size_t na, const void* b, size_t nb)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}


}  // namespace

extern "C" int rdc_step_noalloc(rdc_grid g, const rdc_params* p, const void* u_in,
                                const void* v_in, const void* phi, void* u_out,
                                void* v_out, size_t pitch_bytes, int64_t n,
                                void* stream, int64_t* first_bad)
{
    using namespace rdc;
    if (first_bad) *first_bad = -1;
    if (g.width < 1 || g.height < 1 || n < 0 || !params_ok(p)) return RDC_EINVAL;
    const void* ptrs[5] = {u_in, v_in, phi, u_out, v_out};
    for (const void* q : ptrs)
        if (!q || ((uintptr_t)q % 16)) return RDC_EINVAL;
    const int prec = p->precision;
    const size_t esz = (size_t)state_bytes(prec);
    if (pitch_bytes % 16 || pitch_bytes % esz || pitch_bytes < (size_t)g.width * esz)
        return RDC_EINVAL;
    // The kernels read their inputs through restrict-qualified pointers and
    // write whole output planes, so an output that shares any byte with
    // another buffer would give wrong states: refuse it.  Each state plane
    // spans pitch_bytes * H bytes, phi the same rows at its own element size.
    const size_t sbytes = pitch_bytes * (size_t)g.height;
    const size_t pbytes = pitch_bytes / esz * (prec == P_F64 ? 8 : 4) * (size_t)g.height;
    if (overlap(u_out, sbytes, v_out, sbytes)) return RDC_EINVAL;
    for (void* o : {u_out, v_out})
        if (overlap(o, sbytes, u_in, sbytes) || overlap(o, sbytes, v_in, sbytes) ||
            overlap(o, sbytes, phi, pbytes))
            return RDC_EINVAL;
    const int k = p->k_block == 0 ? 1 : p->k_block;
    // Launches: n / k of the k-step kernel and n % k single steps.  Only
    // calls of two or more launches keep an intermediate state in the
    // scratch array; those whose two scratch planes do not fit it are
    // refused before anything is enqueued.
    const int64_t L = (k > 1) ? n / k + n % k : n;
    const size_t plane = round256(sbytes);
    if (L >= 2 && kFlagBytes + 2 * plane > kScratchBytes) return RDC_EUNSUPPORTED;

    unsigned char* b = nullptr;
    if (L >= 2 || first_bad) {
        void* base = nullptr;
        int rc = scratch_address(&base);
        if (rc) return rc;
        b = static_cast<unsigned char*>(base);
    }
    unsigned long long* flag = reinterpret_cast<unsigned long long*>(b);
    void* su = L >= 2 ? b + kFlagBytes : nullptr;
    void* sv = L >= 2 ? b + kFlagBytes + plane : nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t pitch = (int64_t)(pitch_bytes / esz);

    ModelD m;
    m.eps = p->eps;
    m.f = p->f;
    m.q = p->q;
    m.Du = p->Du;
    m.dt = p->dt;
    m.inv_dx2 = 1.0 / (p->dx * p->dx);

    // Launch shapes: the library's defaults for a grid of this size.  (Any
    // valid shape gives the same bits.)
    const int vec = vec_cells(prec);
    const int64_t vecs = (g.width + vec - 1) / vec;
    int bx = 128;
    if (vecs < bx) bx = (int)(vecs <= 32 ? 32 : (vecs + 31) / 32 * 32);
    const int64_t ncb = (vecs + bx - 1) / bx;
    int rows = 32;
    while (rows > 4 && ncb * ((g.height + rows - 1) / rows) < 152 * 8) rows /= 2;
    const Shape1 s1{bx, rows};
    const ShapeK sk = prec == P_F64 ? ShapeK{32, 32, k, 256} : ShapeK{64, 32, k, 256};

    if (n == 0) {
        cudaError_t e = cudaMemcpy2DAsync(u_out, pitch_bytes, u_in, pitch_bytes,
                                          (size_t)g.width * esz, g.height,
                                          cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(v_out, pitch_bytes, v_in, pitch_bytes,
                                  (size_t)g.width * esz, g.height, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_error();
    } else {
        // Launch j of L writes the output buffers when L - j is even and the
        // scratch pair otherwise, so the last launch lands in the output.
        const void* cu = u_in;
        const void* cv = v_in;
        int64_t left = n;
        for (int64_t j = 1; j <= L; ++j) {
            const bool to_out = ((L - j) % 2) == 0;
            void* du = to_out ? u_out : su;
            void* dv = to_out ? v_out : sv;
            Planes pl{cu, cv, phi, du, dv, g.width, g.height, pitch};
            cudaError_t e;
            if (k > 1 && left >= k) {
                e = launch_stepk(prec, p->flags, pl, m, sk, st);
                left -= k;
            } else {
                e = launch_step1(prec, p->flags, pl, m, s1, st);
                left -= 1;
            }
            if (e != cudaSuccess) return cuda_error();
            cu = du;
            cv = dv;
        }
    }

    if (!first_bad) return RDC_OK;
    // Health check of the output; the flag must start at its sentinel (all
    // ones) on every call because the array keeps the previous call's value.
    cudaError_t e = cudaMemsetAsync(flag, 0xFF, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = launch_health(prec, u_out, g.width, g.height, pitch, p->q, flag, st);
    unsigned long long h = ~0ull;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error();
    if (h != ~0ull) {
        *first_bad = (int64_t)h;
        return RDC_ENONFINITE;
    }
    return RDC_OK;
}
