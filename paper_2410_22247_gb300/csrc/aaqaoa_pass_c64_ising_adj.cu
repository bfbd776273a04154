// Instantiations of the pass kernel for complex64 adjoint passes of Ising plans
// (phi and lambda), in a unit of
// their own so that the pass instantiations compile in parallel.
#include "aaqaoa_pass.cuh"

namespace aaq {

int launch_pass_c64_ising_adj(const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid, cudaStream_t st)
{
    return launch_pass_ising_t<float, 2>(m0, m1, a, grid, st);
}

}  // namespace aaq
