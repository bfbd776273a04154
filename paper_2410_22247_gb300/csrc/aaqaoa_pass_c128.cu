// Instantiations of the pass kernel for complex128 (cut-function and Ising plans,
// forward and adjoint), in a unit of
// their own so that the pass instantiations compile in parallel.
#include "aaqaoa_pass.cuh"

namespace aaq {

int launch_pass_c128(int nv_kernel, const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid,
                     cudaStream_t st)
{
    if (a.icost)
        return nv_kernel == 2 ? launch_pass_ising_t<double, 2>(m0, m1, a, grid, st)
                              : launch_pass_ising_t<double, 1>(m0, m1, a, grid, st);
    return nv_kernel == 2 ? launch_pass_cut_t<double, 2>(m0, m1, a, grid, st)
                          : launch_pass_cut_t<double, 1>(m0, m1, a, grid, st);
}

}  // namespace aaq
