// Step kernels instantiated for __nv_bfloat16 storage of u and v.
#include "rdc_step_impl.cuh"
#include "rdc_stream_impl.cuh"

namespace rdc {

cudaError_t launch_step1_bf16(int mode, const Planes& g, const ModelD& m, Shape1 s, cudaStream_t st)
{
    return launch_step1_t<__nv_bfloat16>(mode, g, m, s, st);
}

cudaError_t launch_stepk_bf16(int mode, const Planes& g, const ModelD& m, ShapeK s, cudaStream_t st)
{
    return launch_stepk_t<__nv_bfloat16>(mode, g, m, s, st);
}

size_t stepk_smem_bf16(ShapeK s) { return stepk_smem_t<__nv_bfloat16>(s); }

cudaError_t launch_stream_bf16(const Planes& g, const ModelD& m, int k, int rows, cudaStream_t st)
{
    return launch_stream_t<__nv_bfloat16>(g, m, k, rows, st);
}

cudaError_t launch_batch_step1_bf16(const GridDesc* d, const TileMap* map, int rows,
    unsigned* queue, int j, long long sbase, int sr, int ctas, cudaStream_t st)
{
    return launch_batch_step1_t<__nv_bfloat16>(d, map, rows, queue, j, sbase, sr, ctas, st);
}

cudaError_t launch_batch_stream_bf16(const GridDesc* d, const TileMap* map, int rows,
    unsigned* queue, int k, int j, long long sbase, int sr, int ctas, cudaStream_t st)
{
    return launch_batch_stream_t<__nv_bfloat16>(d, map, rows, queue, k, j, sbase, sr, ctas, st);
}

int batch_stream_outc_bf16(int k, bool sr) { return stream_outc_t<__nv_bfloat16>(k, sr); }

}  // namespace rdc
