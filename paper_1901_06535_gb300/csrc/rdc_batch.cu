// Batches of independent grids (parameter sweeps, many sessions): one device
// allocation per grid (grids can join and leave), a device table of grid
// descriptors, persistent launches whose warps take warp-sized work items of
// all grids from a queue, CUDA graphs of whole step sequences, and an
// autotuner for the launch shape.
//
// Grids join and leave without stalling the host: their memory, the work
// lists and the descriptor table come from the batch's own stream-ordered
// memory pool (cudaMallocFromPoolAsync / cudaFreeAsync on the batch's
// stream, memory kept in the pool for reuse), and every upload is an
// asynchronous copy on that stream, so rdc_batch_add, rdc_batch_remove and
// the work-list rebuild they cause enqueue work behind the frames in flight
// instead of waiting for them (a serving loop keeps polling other streams
// meanwhile).
//
// Each grid in a batch runs the same cell_update as a single simulation with
// the same parameters, so a grid's result is bit-identical whether it is
// stepped alone, in a batch, or in any subset of one.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "rdc.h"
#include "rdc_host.h"
#include "rdc_internal.h"

using namespace rdc;

namespace {

const double kPhiActive = 0.054;  // Table 1

struct Config {
    int k = 1;       // Euler steps per launch
    int rows = 16;   // rows per item, single-step kernel
    int krows = 64;  // rows per item, streamed k-step kernel
};

// A tile map on the device (see TileMap) with room for `cap` grids, and the
// host copy it was uploaded from.
struct MapBuf {
    TileMap* dev = nullptr;
    int cap = 0;
    std::vector<int> host;
    int total = 0;          // tiles of the map as last built
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
};

}  // namespace

struct rdc_batch {
    int n = 0;                       // slots (live or free)
    int prec = 0;
    int k_block = 0;
    int sr = 0;                      // RDC_STOCH_ROUND on every grid
    std::vector<rdc_grid> grids;
    std::vector<rdc_params> params;
    std::vector<GridDesc> desc;      // host copy; par kept current
    std::vector<void*> mem;          // per-slot allocation (nullptr = free slot)
    cudaMemPool_t pool = nullptr;    // stream-ordered pool of every device buffer below
    std::vector<double> phi_max;     // per slot: largest phi of the grid's map
    GridDesc* d_desc = nullptr;
    int d_desc_cap = 0;
    unsigned long long* d_flag = nullptr;  // health flag at +0, work queue at +64
    void* stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    Config cfg;
    bool use_graphs = true;
    // tile maps of the single-step and the k-step kernel, rebuilt for the
    // grids of every call at fixed device addresses, and graphs of launch
    // sequences keyed by (n, k, rows, krows), valid for any subset
    MapBuf map1, mapk;
    std::map<std::vector<int64_t>, GraphEntry> graphs;
    int64_t launches = 0;
    int64_t graph_launches = 0;
    double cells_stepped = 0.0;
};

namespace {

// Stream-ordered allocation from the batch's pool: usable by work enqueued on
// the batch's stream after this call; no synchronisation.
cudaError_t dev_alloc(rdc_batch* b, void** p, size_t bytes)
{
    return cudaMallocFromPoolAsync(p, bytes, b->pool, b->stream);
}

// Stream-ordered free: the memory returns to the pool once the work enqueued
// on the batch's stream before it has finished.
void dev_free(rdc_batch* b, void* p)
{
    if (p) cudaFreeAsync(p, b->stream);
}

void release_map(rdc_batch* b, MapBuf& M)
{
    dev_free(b, M.dev);
    M.dev = nullptr;
    M.cap = 0;
}

void free_graphs(rdc_batch* b)
{
    for (auto& kv : b->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    b->graphs.clear();
}

int persistent_ctas(int64_t ntiles)
{
    // 128-thread CTAs, 4 warps each; enough CTAs to fill every SM with as
    // many as fit (warps take tiles from a shared queue, so CTAs beyond that
    // find it empty and end at once), never more than the tiles need
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = sms * 8;
    const int64_t need = (ntiles + 3) / 4;
    return (int)std::max<int64_t>(1, std::min(want, need));
}

// The two counters of the batched kernels' work queue (zero between launches).
unsigned* queue_of(rdc_batch* b) { return reinterpret_cast<unsigned*>(b->d_flag) + 16; }

// Tiles of `cols` x `rows` cells of grid g.
int64_t grid_tiles(const rdc_batch* b, int g, int cols, int rows, int* tiles_x)
{
    const int W = b->grids[g].width, H = b->grids[g].height;
    *tiles_x = (W + cols - 1) / cols;
    return (int64_t)*tiles_x * ((H + rows - 1) / rows);
}

// Builds the tile map of `grids` for tiles of `cols` x `rows` cells and
// enqueues its upload on the batch's stream (behind the launches that still
// read the previous map; a pageable source is staged before the call
// returns).  The device buffer keeps its address unless it must grow, which
// invalidates the captured graphs.
int build_map(rdc_batch* b, const std::vector<int>& grids, int cols, int rows, MapBuf& M)
{
    if (cols <= 0 || rows <= 0) return RDC_EINVAL;
    const int ns = (int)grids.size();
    std::vector<int>& h = M.host;
    h.assign(4 + 4 * (size_t)std::max(ns, 1), 0);
    int64_t total = 0;
    for (int i = 0; i < ns; ++i) {
        int tx = 0;
        const int64_t t = grid_tiles(b, grids[i], cols, rows, &tx);
        h[4 + 4 * i] = grids[i];
        h[4 + 4 * i + 1] = tx;
        h[4 + 4 * i + 2] = (int)total;
        total += t;
    }
    if (total > INT_MAX) return RDC_EUNSUPPORTED;
    h[0] = ns;
    h[1] = (int)total;
    M.total = (int)total;
    const int need = std::max(ns, 1);
    if (M.cap < need) {
        release_map(b, M);
        const int cap = std::max(16, 2 * std::max(need, b->n));
        cudaError_t e = dev_alloc(b, (void**)&M.dev, sizeof(int) * (4 + 4 * (size_t)cap));
        if (e != cudaSuccess) return host_cuda_fail(e, "cudaMallocFromPoolAsync(tile map)");
        M.cap = cap;
        free_graphs(b);  // graphs captured the old map's address
    }
    cudaError_t e = cudaMemcpyAsync(M.dev, h.data(), sizeof(int) * h.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    return e == cudaSuccess ? RDC_OK : host_cuda_fail(e, "cudaMemcpyAsync(tile map)");
}

// Tile maps of both kernels for the grids of a call.
int build_maps(rdc_batch* b, const std::vector<int>& grids)
{
    int rc = build_map(b, grids, batch_step1_cols(b->prec), b->cfg.rows, b->map1);
    if (rc == RDC_OK && b->cfg.k > 1)
        rc = build_map(b, grids, batch_stream_outc(b->prec, b->cfg.k, b->sr != 0), b->cfg.krows, b->mapk);
    return rc;
}

// Tiles of every live grid for the current shape (kernel k > 1: streamed).
int64_t live_tiles(const rdc_batch* b, bool streamed)
{
    const int cols = streamed ? batch_stream_outc(b->prec, b->cfg.k, b->sr != 0) : batch_step1_cols(b->prec);
    const int rows = streamed ? b->cfg.krows : b->cfg.rows;
    int64_t t = 0;
    for (int g = 0; g < b->n; ++g) {
        int tx = 0;
        if (b->mem[g]) t += grid_tiles(b, g, cols, rows, &tx);
    }
    return t;
}

// Enqueues the launch sequence of n steps for the subset: n / k streamed
// k-step launches, then n % k single steps; launch j reads buffer
// (par + j) & 1 of each grid.
int enqueue_sequence(rdc_batch* b, int64_t n, int ctas1, int ctask, int64_t* launches)
{
    const int k = b->cfg.k;
    int64_t j = 0, left = n;
    while (left > 0) {
        cudaError_t e;
        const long long sbase = (long long)(n - left);  // steps of this call already enqueued
        if (k > 1 && left >= k) {
            e = launch_batch_stream(b->prec, b->d_desc, b->mapk.dev, b->cfg.krows, queue_of(b),
                                    k, (int)(j & 1), sbase, b->sr, ctask, b->stream);
            left -= k;
        } else {
            e = launch_batch_step1(b->prec, b->d_desc, b->map1.dev, b->cfg.rows, queue_of(b),
                                   (int)(j & 1), sbase, b->sr, ctas1, b->stream);
            left -= 1;
        }
        if (e != cudaSuccess) return host_cuda_fail(e, "batched step kernel");
        ++j;
    }
    *launches = j;
    return RDC_OK;
}

int upload_desc(rdc_batch* b)
{
    if (b->n == 0) return RDC_OK;
    if (b->d_desc_cap < b->n) {
        dev_free(b, b->d_desc);   // after the launches that still read it
        b->d_desc = nullptr;
        b->d_desc_cap = 0;
        const int cap = std::max(16, 2 * b->n);
        cudaError_t e = dev_alloc(b, (void**)&b->d_desc, sizeof(GridDesc) * cap);
        if (e != cudaSuccess) return host_cuda_fail(e, "cudaMallocFromPoolAsync(descriptors)");
        b->d_desc_cap = cap;
        free_graphs(b);  // graphs captured the old table's address
    }
    cudaError_t e = cudaMemcpyAsync(b->d_desc, b->desc.data(), b->desc.size() * sizeof(GridDesc),
                                    cudaMemcpyHostToDevice, b->stream);
    return e == cudaSuccess ? RDC_OK : host_cuda_fail(e, "cudaMemcpyAsync(descriptors)");
}

// Staging buffer for type conversions of host data (stream-ordered, so the
// old buffer is released only after the work that still uses it).
int ensure_stage(rdc_batch* b, size_t bytes)
{
    if (b->stage_bytes >= bytes) return RDC_OK;
    dev_free(b, b->stage);
    b->stage = nullptr;
    b->stage_bytes = 0;
    cudaError_t e = dev_alloc(b, &b->stage, bytes);
    if (e != cudaSuccess) return host_cuda_fail(e, "cudaMallocFromPoolAsync(stage)");
    b->stage_bytes = bytes;
    return RDC_OK;
}

// Allocates and initialises one grid in slot g (rest state of its phi map).
// Everything is enqueued on the batch's stream; nothing waits for the device.
int init_slot(rdc_batch* b, int g, rdc_grid grid, const rdc_params& p, const float* phi_host)
{
    const int prec = b->prec;
    const int esz = state_bytes(prec), psz = phi_bytes(prec);
    auto r256 = [](size_t x) { return (x + 255) / 256 * 256; };
    const int64_t pitch = (grid.width + 63) / 64 * 64;
    const size_t sp = r256((size_t)pitch * grid.height * esz);
    const size_t total = 4 * sp + r256((size_t)pitch * grid.height * psz);
    void* mem = nullptr;
    cudaError_t e = dev_alloc(b, &mem, total);
    if (e != cudaSuccess) return host_cuda_fail(e, "cudaMallocFromPoolAsync(batch grid)");
    e = cudaMemsetAsync(mem, 0, total, b->stream);
    GridDesc d;
    std::memset(&d, 0, sizeof d);
    unsigned char* q = (unsigned char*)mem;
    d.u[0] = q;
    d.u[1] = q + sp;
    d.v[0] = q + 2 * sp;
    d.v[1] = q + 3 * sp;
    d.phi = q + 4 * sp;
    d.W = grid.width;
    d.H = grid.height;
    d.pitch = pitch;
    d.eps = p.eps;
    d.f = p.f;
    d.q = p.q;
    d.Du = p.Du;
    d.dt = p.dt;
    d.inv_dx2 = 1.0 / (p.dx * p.dx);
    d.par = 0;
    d.seed = (unsigned)p.round_seed;
    d.steps = 0;
    if (e == cudaSuccess) {
        if (phi_host && psz == (int)sizeof(float)) {
            // float maps go straight into the pitched plane (from pinned host
            // memory this copy does not involve the host at all)
            e = cudaMemcpy2DAsync((void*)d.phi, (size_t)pitch * psz, phi_host,
                                  (size_t)grid.width * sizeof(float),
                                  (size_t)grid.width * sizeof(float), grid.height,
                                  cudaMemcpyHostToDevice, b->stream);
        } else if (phi_host) {
            const size_t bytes = (size_t)grid.width * grid.height * sizeof(float);
            int rc = ensure_stage(b, bytes);
            if (rc) {
                dev_free(b, mem);
                return rc;
            }
            e = cudaMemcpyAsync(b->stage, phi_host, bytes, cudaMemcpyHostToDevice, b->stream);
            if (e == cudaSuccess)
                e = launch_phi_in(prec, 0, b->stage, (void*)d.phi, d.W, d.H, pitch, b->stream);
        } else {
            e = launch_fill_phi(prec, (void*)d.phi, d.W, d.H, pitch, kPhiActive, b->stream);
        }
    }
    if (e == cudaSuccess)
        e = launch_rest(prec, d.u[0], d.v[0], d.phi, d.W, d.H, pitch, p.f, p.q, b->stream);
    if (e != cudaSuccess) {
        dev_free(b, mem);
        return host_cuda_fail(e, "batch grid initialisation");
    }
    b->grids[g] = grid;
    b->params[g] = p;
    b->desc[g] = d;
    b->mem[g] = mem;
    return RDC_OK;
}

bool grid_ok(const rdc_batch* b, rdc_grid grid, const rdc_params* p, const float* phi_host,
             double* phi_max)
{
    if (grid.width < 1 || grid.height < 1 || !host_params_valid(p)) return false;
    if (p->precision != b->prec || p->flags != (b->sr ? RDC_STOCH_ROUND : 0)) return false;
    *phi_max = kPhiActive;
    if (phi_host)
        return host_scan_phi(phi_host, 0, (int64_t)grid.width * grid.height, p, phi_max);
    return host_phi_ok(kPhiActive, p);
}

bool subset_of(rdc_batch* b, const int32_t* idx, int32_t m, std::vector<int>* out)
{
    out->clear();
    if (!idx) {
        for (int g = 0; g < b->n; ++g)
            if (b->mem[g]) out->push_back(g);
        return true;
    }
    if (m < 0) return false;
    for (int32_t i = 0; i < m; ++i) {
        if (idx[i] < 0 || idx[i] >= b->n || !b->mem[idx[i]]) return false;
        out->push_back(idx[i]);
    }
    std::sort(out->begin(), out->end());
    return std::adjacent_find(out->begin(), out->end()) == out->end();
}

}  // namespace

extern "C" {

int rdc_batch_create(int32_t n, const rdc_grid* grids, const rdc_params* params,
                     const float* const* phi_host, void* stream, rdc_batch** out)
{
    if (!out) return RDC_EINVAL;
    *out = nullptr;
    if (n < 0 || !params || (n > 0 && !grids)) return RDC_EINVAL;
    if (!host_params_valid(&params[0]) || (params[0].flags & ~RDC_STOCH_ROUND) != 0)
        return RDC_EINVAL;
    int rc = host_check_device();
    if (rc) return rc;
    rdc_batch* b = new (std::nothrow) rdc_batch();
    if (!b) return RDC_ENOMEM;
    b->prec = params[0].precision;
    b->k_block = params[0].k_block;
    b->sr = (params[0].flags & RDC_STOCH_ROUND) ? 1 : 0;
    b->cfg.k = b->k_block == 0 ? 1 : b->k_block;
    for (int g = 0; g < n; ++g) {
        double mx = 0.0;
        if (params[g].k_block != b->k_block ||
            !grid_ok(b, grids[g], &params[g], phi_host ? phi_host[g] : nullptr, &mx)) {
            delete b;
            return RDC_EINVAL;
        }
    }
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return host_cuda_fail(e, "cudaStreamCreateWithFlags");
        }
        b->owns_stream = true;
    }
    // the stream-ordered pool that grids, work lists and tables come from;
    // freed memory stays in it for the next grid instead of going back to
    // the driver
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&b->pool, &props);
    }
    if (e == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(b->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e != cudaSuccess) {
        rdc_batch_destroy(b);
        return host_cuda_fail(e, "cudaMemPoolCreate");
    }
    e = cudaMalloc((void**)&b->d_flag, 256);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_flag, 0, 256, b->stream);  // queue zeroed
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        rdc_batch_destroy(b);
        return host_cuda_fail(e, "cudaMalloc(flag)");
    }
    for (int g = 0; g < n; ++g) {
        int32_t idx = -1;
        rc = rdc_batch_add(b, grids[g], &params[g], phi_host ? phi_host[g] : nullptr, &idx);
        if (rc) {
            rdc_batch_destroy(b);
            return rc;
        }
    }
    *out = b;
    return RDC_OK;
}

int rdc_batch_add(rdc_batch* b, rdc_grid grid, const rdc_params* p, const float* phi_host,
                  int32_t* idx)
{
    NvtxRange nvtx("rdc_batch_add");
    if (!b || !idx || !p) return RDC_EINVAL;
    *idx = -1;
    double mx = 0.0;
    if (p->k_block != b->k_block || !grid_ok(b, grid, p, phi_host, &mx)) return RDC_EINVAL;
    int g = 0;
    while (g < b->n && b->mem[g]) ++g;  // reuse a free slot
    if (g == b->n) {
        b->grids.push_back(grid);
        b->params.push_back(*p);
        b->desc.push_back(GridDesc{});
        b->mem.push_back(nullptr);
        b->phi_max.push_back(0.0);
        b->n += 1;
    }
    int rc = init_slot(b, g, grid, *p, phi_host);
    if (rc) return rc;
    b->phi_max[g] = mx;
    free_graphs(b);  // their CTA counts were sized for the previous grids
    *idx = g;
    return RDC_OK;
}

int rdc_batch_remove(rdc_batch* b, int32_t idx)
{
    NvtxRange nvtx("rdc_batch_remove");
    if (!b || idx < 0 || idx >= b->n || !b->mem[idx]) return RDC_EINVAL;
    // returned to the pool behind the work already enqueued for it; the slot
    // can take a new grid at once
    dev_free(b, b->mem[idx]);
    b->mem[idx] = nullptr;
    std::memset(&b->desc[idx], 0, sizeof(GridDesc));
    free_graphs(b);
    return RDC_OK;
}

void rdc_batch_destroy(rdc_batch* b)
{
    if (!b) return;
    free_graphs(b);
    if (b->pool) {
        release_map(b, b->map1);
        release_map(b, b->mapk);
        for (void* m : b->mem) dev_free(b, m);
        dev_free(b, b->d_desc);
        dev_free(b, b->stage);
    }
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->pool) cudaMemPoolDestroy(b->pool);
    if (b->d_flag) cudaFree(b->d_flag);
    if (b->owns_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int rdc_batch_seed(rdc_batch* b, int32_t idx, double cx, double cy, double r, double value)
{
    if (!b || idx < 0 || idx >= b->n || !b->mem[idx] || !std::isfinite(cx) || !std::isfinite(cy) ||
        !std::isfinite(value) || !(r >= 0.0) || !(r < 16777216.0))
        return RDC_EINVAL;
    const GridDesc& d = b->desc[idx];
    cudaError_t e = launch_seed(b->prec, d.u[d.par], d.W, d.H, d.pitch, cx, cy, r, value, b->stream);
    return e == cudaSuccess ? RDC_OK : host_cuda_fail(e, "seed kernel");
}

int rdc_batch_set_state(rdc_batch* b, int32_t idx, const void* u_host, const void* v_host,
                        int32_t dtype)
{
    if (!b || idx < 0 || idx >= b->n || !b->mem[idx] || dtype < 0 || dtype > 3)
        return RDC_EINVAL;
    const GridDesc& d = b->desc[idx];
    const int esz = state_bytes(b->prec);
    const void* src[2] = {u_host, v_host};
    void* dst[2] = {d.u[d.par], d.v[d.par]};
    for (int k = 0; k < 2; ++k) {
        if (!src[k]) continue;
        cudaError_t e;
        if (dtype == b->prec) {
            e = cudaMemcpy2DAsync(dst[k], (size_t)d.pitch * esz, src[k], (size_t)d.W * esz,
                                  (size_t)d.W * esz, d.H, cudaMemcpyHostToDevice, b->stream);
        } else {
            const size_t bytes = (size_t)d.W * d.H * dtype_bytes(dtype);
            const int rc = ensure_stage(b, bytes);
            if (rc) return rc;
            e = cudaMemcpyAsync(b->stage, src[k], bytes, cudaMemcpyHostToDevice, b->stream);
            if (e == cudaSuccess)
                e = launch_pack_in(b->prec, dtype, b->stage, dst[k], d.W, d.H, d.pitch, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        }
        if (e != cudaSuccess) return host_cuda_fail(e, "rdc_batch_set_state");
    }
    return RDC_OK;
}

int rdc_batch_set_step_index(rdc_batch* b, int32_t idx, int64_t n)
{
    if (!b || idx < 0 || idx >= b->n || !b->mem[idx] || n < 0) return RDC_EINVAL;
    b->desc[idx].steps = n;  // uploaded with the descriptors at the next step
    return RDC_OK;
}

int rdc_batch_step(rdc_batch* b, const int32_t* idx, int32_t m, int64_t n)
{
    NvtxRange nvtx("rdc_batch_step");
    if (!b || n < 0) return RDC_EINVAL;
    std::vector<int> subset;
    if (!subset_of(b, idx, m, &subset)) return RDC_EINVAL;
    if (subset.empty() || n == 0) return RDC_OK;
    for (int g = 0; g < b->n; ++g) b->desc[g].active = 0;
    for (int g : subset) b->desc[g].active = 1;
    int rc = upload_desc(b);
    if (rc) return rc;
    // the tile maps of this call's grids, outside any capture (they may
    // allocate); a captured graph reads them at their fixed addresses
    if ((rc = build_maps(b, subset))) return rc;
    int64_t L = 0;
    if (b->use_graphs) {
        // a graph serves every subset, so its persistent launches are sized
        // for all live grids (CTAs beyond the call's tiles find the queue
        // empty and end at once)
        const int ctas1 = persistent_ctas(live_tiles(b, false));
        const int ctask = b->cfg.k > 1 ? persistent_ctas(live_tiles(b, true)) : 1;
        const std::vector<int64_t> key{n, b->cfg.k, b->cfg.rows, b->cfg.krows};
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return host_cuda_fail(e, "cudaStreamBeginCapture");
            rc = enqueue_sequence(b, n, ctas1, ctask, &L);
            e = cudaStreamEndCapture(b->stream, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return host_cuda_fail(e, "cudaStreamEndCapture");
            GraphEntry ge;
            e = cudaGraphInstantiate(&ge.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return host_cuda_fail(e, "cudaGraphInstantiate");
            ge.launches = L;
            if (b->graphs.size() >= 64) free_graphs(b);
            it = b->graphs.emplace(key, ge).first;
        }
        cudaError_t e;
        {
            NvtxRange replay("rdc_batch_step: graph replay");
            e = cudaGraphLaunch(it->second.exec, b->stream);
        }
        if (e != cudaSuccess) return host_cuda_fail(e, "cudaGraphLaunch");
        L = it->second.launches;
        b->graph_launches += 1;
    } else {
        rc = enqueue_sequence(b, n, persistent_ctas(b->map1.total),
                              b->cfg.k > 1 ? persistent_ctas(b->mapk.total) : 1, &L);
        if (rc) return rc;
    }
    for (int g : subset) {
        b->desc[g].par = (int)((b->desc[g].par + L) & 1);
        b->desc[g].steps += n;
        b->cells_stepped += (double)b->grids[g].width * b->grids[g].height * (double)n;
    }
    b->launches += L;
    return RDC_OK;
}

int rdc_batch_check(rdc_batch* b, int32_t idx, int64_t* first_bad)
{
    if (!b || idx < 0 || idx >= b->n || !b->mem[idx]) return RDC_EINVAL;
    const GridDesc& d = b->desc[idx];
    cudaError_t e = cudaMemsetAsync(b->d_flag, 0xFF, sizeof(unsigned long long), b->stream);
    if (e == cudaSuccess)
        e = launch_health(b->prec, d.u[d.par], d.W, d.H, d.pitch, b->params[idx].q, b->d_flag,
                          b->stream);
    unsigned long long h = ~0ull;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&h, b->d_flag, sizeof h, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return host_cuda_fail(e, "batch health check");
    if (first_bad) *first_bad = (h == ~0ull) ? -1 : (int64_t)h;
    return h == ~0ull ? RDC_OK : RDC_ENONFINITE;
}

int rdc_batch_read(rdc_batch* b, int32_t idx, void* u_out, void* v_out, int32_t dtype)
{
    if (!b || idx < 0 || idx >= b->n || !b->mem[idx] || dtype < 0 || dtype > 3)
        return RDC_EINVAL;
    const GridDesc& d = b->desc[idx];
    const int esz = state_bytes(b->prec);
    const void* src[2] = {d.u[d.par], d.v[d.par]};
    void* dst[2] = {u_out, v_out};
    for (int k = 0; k < 2; ++k) {
        if (!dst[k]) continue;
        cudaError_t e;
        if (dtype == b->prec) {
            e = cudaMemcpy2DAsync(dst[k], (size_t)d.W * esz, src[k], (size_t)d.pitch * esz,
                                  (size_t)d.W * esz, d.H, cudaMemcpyDeviceToHost, b->stream);
        } else {
            const size_t bytes = (size_t)d.W * d.H * dtype_bytes(dtype);
            const int rc = ensure_stage(b, bytes);
            if (rc) return rc;
            e = launch_pack_out(b->prec, dtype, src[k], b->stage, d.W, d.H, d.pitch, b->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(dst[k], b->stage, bytes, cudaMemcpyDeviceToHost, b->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return host_cuda_fail(e, "rdc_batch_read");
    }
    return rdc_batch_check(b, idx, nullptr);
}

int rdc_batch_sync(rdc_batch* b)
{
    if (!b) return RDC_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? RDC_OK : host_cuda_fail(e, "cudaStreamSynchronize");
}

int rdc_batch_set_config(rdc_batch* b, int32_t k, int32_t rows, int32_t krows, int32_t graphs)
{
    if (!b || k < 1 || k > 8 || rows < 1 || krows < 1 || graphs < 0 || graphs > 1)
        return RDC_EINVAL;
    free_graphs(b);
    b->cfg.k = k;
    b->cfg.rows = rows;
    b->cfg.krows = krows;
    b->use_graphs = graphs != 0;
    return RDC_OK;
}

int rdc_batch_get_info(rdc_batch* b, rdc_batch_info* out)
{
    if (!b || !out) return RDC_EINVAL;
    std::memset(out, 0, sizeof *out);
    int live = 0;
    for (void* m : b->mem) live += m ? 1 : 0;
    out->ngrids = live;
    out->slots = b->n;
    out->precision = b->prec;
    out->k = b->cfg.k;
    out->rows = b->cfg.rows;
    out->krows = b->cfg.krows;
    out->graphs = b->use_graphs ? 1 : 0;
    double cells = 0;
    for (int g = 0; g < b->n; ++g)
        if (b->mem[g]) cells += (double)b->grids[g].width * b->grids[g].height;
    out->total_cells = cells;
    out->launches = b->launches;
    out->graph_launches = b->graph_launches;
    out->cells_stepped = b->cells_stepped;
    out->stream = (void*)b->stream;
    return RDC_OK;
}

int rdc_batch_get_grid(rdc_batch* b, int32_t idx, rdc_grid* out)
{
    if (!b || !out || idx < 0 || idx >= b->n || !b->mem[idx]) return RDC_EINVAL;
    *out = b->grids[idx];
    return RDC_OK;
}

int rdc_batch_stability(rdc_batch* b, int32_t idx, double* rho)
{
    if (!b || !rho || idx < 0 || idx >= b->n || !b->mem[idx]) return RDC_EINVAL;
    return host_stability(b->params[idx], b->phi_max[idx], rho);
}

int rdc_batch_tune(rdc_batch* b, int32_t reps, rdc_batch_info* out)
{
    NvtxRange nvtx("rdc_batch_tune");
    if (!b || reps < 1) return RDC_EINVAL;
    double cells = 0;
    std::vector<int> live;
    for (int g = 0; g < b->n; ++g) {
        b->desc[g].active = b->mem[g] ? 1 : 0;
        if (b->mem[g]) {
            cells += (double)b->grids[g].width * b->grids[g].height;
            live.push_back(g);
        }
    }
    if (cells == 0) return RDC_EINVAL;
    int rc = upload_desc(b);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    cudaError_t ee = cudaEventCreate(&e0);
    if (ee != cudaSuccess) return host_cuda_fail(ee, "cudaEventCreate");
    ee = cudaEventCreate(&e1);
    if (ee != cudaSuccess) {
        cudaEventDestroy(e0);
        return host_cuda_fail(ee, "cudaEventCreate");
    }
    const Config saved = b->cfg;
    Config best = saved;
    double best_rate = -1.0;
    struct Cand { int k, rows, krows; };
    std::vector<Cand> cands;
    for (int rows : {8, 16, 32}) cands.push_back({1, rows, saved.krows});
    for (int k : {2, 3, 4, 5, 6, 8})
        for (int krows : {32, 64, 128, 256}) cands.push_back({k, saved.rows, krows});
    for (const Cand& c : cands) {
        b->cfg.k = c.k;
        b->cfg.rows = c.rows;
        b->cfg.krows = c.krows;
        rc = build_maps(b, live);
        if (rc) break;
        // Every timed launch reads the current buffers (j = 0) and writes the
        // spare ones, so tuning never advances the state.
        auto launch = [&]() {
            return c.k > 1 ? launch_batch_stream(b->prec, b->d_desc, b->mapk.dev, c.krows,
                                                 queue_of(b), c.k, 0, 0, b->sr,
                                                 persistent_ctas(b->mapk.total), b->stream)
                           : launch_batch_step1(b->prec, b->d_desc, b->map1.dev, c.rows,
                                                queue_of(b), 0, 0, b->sr,
                                                persistent_ctas(b->map1.total), b->stream);
        };
        cudaError_t e = launch();  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = host_cuda_fail(e, "autotune launch");
            break;
        }
        const double rate = cells * c.k * reps / (ms * 1e-3);
        if (rate > best_rate) {
            best_rate = rate;
            best = b->cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    free_graphs(b);
    b->cfg = rc ? saved : best;
    if (rc) return rc;
    if (out) {
        rdc_batch_get_info(b, out);
        out->tuned_gcups = best_rate / 1e9;
    }
    return RDC_OK;
}

}  // extern "C"
