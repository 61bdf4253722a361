// ptg_opensimplex3d_f16_dyadic.cu -- the FP16 instance of the 3D OpenSimplex-style
// generator (ptg_opensimplex3d.cuh) for fields whose every octave step is a power of two.
#include "ptg_opensimplex3d.cuh"

namespace ptg {

cudaError_t launch_opensimplex3d_f16_dyadic(const Simplex3Plan& P, cudaStream_t stream)
{
    return launch_instance<__half, true>(P, stream);
}

}  // namespace ptg
