// ptg_opensimplex3d_f16.cu -- the FP16 instance of the 3D OpenSimplex-style
// generator (ptg_opensimplex3d.cuh) for fields with any frequency ratio.
#include "ptg_opensimplex3d.cuh"

namespace ptg {

cudaError_t launch_opensimplex3d_f16(const Simplex3Plan& P, cudaStream_t stream)
{
    return launch_instance<__half, false>(P, stream);
}

}  // namespace ptg
