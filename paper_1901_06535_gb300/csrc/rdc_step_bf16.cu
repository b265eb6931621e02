// Step kernels instantiated for __nv_bfloat16 storage of u and v.
#include "rdc_step_impl.cuh"

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

}  // namespace rdc
