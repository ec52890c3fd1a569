// batch_stage3.cu -- instantiations of the batched row kernels (group 3);
// the groups compile in parallel.
#include "batch_stage.cuh"

namespace xamg {

int launch_bk_g3(int kind, int nv, int opt, const void *params, const int *sel, int grid,
                 cudaStream_t st) {
  switch (kind) {
    case BK_F_XLAST_DOT2: return bk_launch_t<BK_F_XLAST_DOT2>(nv, opt, params, sel, grid, st);
    case BK_D_YDOT: return bk_launch_t<BK_D_YDOT>(nv, opt, params, sel, grid, st);
    case BK_D_YDOT2: return bk_launch_t<BK_D_YDOT2>(nv, opt, params, sel, grid, st);
    default: return -2;
  }
}

}  // namespace xamg
