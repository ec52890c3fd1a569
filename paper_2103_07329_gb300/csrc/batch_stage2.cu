// batch_stage2.cu -- instantiations of the batched row kernels (group 2);
// the groups compile in parallel.
#include "batch_stage.cuh"

namespace xamg {

int launch_bk_g2(int kind, int nv, int opt, const void *params, const int *sel, int grid,
                 cudaStream_t st) {
  switch (kind) {
    case BK_F_Y_POS: return bk_launch_t<BK_F_Y_POS>(nv, opt, params, sel, grid, st);
    case BK_F_D0_NEG: return bk_launch_t<BK_F_D0_NEG>(nv, opt, params, sel, grid, st);
    case BK_F_XLAST: return bk_launch_t<BK_F_XLAST>(nv, opt, params, sel, grid, st);
    default: return -2;
  }
}

}  // namespace xamg
