// Step kernels instantiated for float storage of u and v.
#include "rdc_step_impl.cuh"

namespace rdc {

cudaError_t launch_step1_f32(int mode, const Planes& g, const ModelD& m, Shape1 s, cudaStream_t st)
{
    return launch_step1_t<float>(mode, g, m, s, st);
}

cudaError_t launch_stepk_f32(int mode, const Planes& g, const ModelD& m, ShapeK s, cudaStream_t st)
{
    return launch_stepk_t<float>(mode, g, m, s, st);
}

size_t stepk_smem_f32(ShapeK s) { return stepk_smem_t<float>(s); }

}  // namespace rdc
