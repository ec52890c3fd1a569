// batch_stage1.cu -- instantiations of the batched row kernels (group 1);
// the groups compile in parallel.
#include "batch_stage.cuh"

namespace xamg {

int launch_bk_g1(int kind, int nv, int opt, const void *params, const int *sel, int grid,
                 cudaStream_t st) {
  switch (kind) {
    case BK_F_YDN: return bk_launch_t<BK_F_YDN>(nv, opt, params, sel, grid, st);
    case BK_F_YXDP: return bk_launch_t<BK_F_YXDP>(nv, opt, params, sel, grid, st);
    case BK_F_D0_POS: return bk_launch_t<BK_F_D0_POS>(nv, opt, params, sel, grid, st);
    default: return -2;
  }
}

}  // namespace xamg
