// ptg_opensimplex3d_f32.cu -- the FP32 instance of the 3D OpenSimplex-style
// generator (ptg_opensimplex3d.cuh) for fields with any frequency ratio, and
// the dispatch over the four instances.
#include "ptg_opensimplex3d.cuh"

namespace ptg {

cudaError_t launch_opensimplex3d_f32(const Simplex3Plan& P, cudaStream_t stream)
{
    return launch_instance<float, false>(P, stream);
}

// Fields whose every octave step is a power of two take the instance that
// compiles only the exact-offset octave code.
cudaError_t launch_opensimplex3d(const Simplex3Plan& P, cudaStream_t stream)
{
    const bool all_exact = P.exact_mask == (P.N >= 32 ? 0xffffffffu : (1u << P.N) - 1u);
    if (P.dtype == 1) return all_exact ? launch_opensimplex3d_f16_dyadic(P, stream) : launch_opensimplex3d_f16(P, stream);
    return all_exact ? launch_opensimplex3d_f32_dyadic(P, stream) : launch_opensimplex3d_f32(P, stream);
}

}  // namespace ptg
