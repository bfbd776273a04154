// Instantiations of the pass kernel for complex64 forward passes of cut-function
// plans (one statevector), in a unit of
// their own so that the pass instantiations compile in parallel.
#include "aaqaoa_pass.cuh"

namespace aaq {

int launch_pass_c64_fwd(const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid, cudaStream_t st)
{
    return launch_pass_cut_t<float, 1>(m0, m1, a, grid, st);
}

}  // namespace aaq
