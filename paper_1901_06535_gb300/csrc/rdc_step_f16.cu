// Step kernels instantiated for __half storage of u and v.
#include "rdc_step_impl.cuh"

namespace rdc {

cudaError_t launch_step1_f16(int mode, const Planes& g, const ModelD& m, Shape1 s, cudaStream_t st)
{
    return launch_step1_t<__half>(mode, g, m, s, st);
}

cudaError_t launch_stepk_f16(int mode, const Planes& g, const ModelD& m, ShapeK s, cudaStream_t st)
{
    return launch_stepk_t<__half>(mode, g, m, s, st);
}

size_t stepk_smem_f16(ShapeK s) { return stepk_smem_t<__half>(s); }

}  // namespace rdc
