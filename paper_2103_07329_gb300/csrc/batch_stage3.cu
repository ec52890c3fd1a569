// batch_stage3.cu -- instantiations of the batched row stages (group 3);
// the groups compile in parallel.
#include <algorithm>

#include "batch_stage.cuh"

namespace xamg {

int launch_bstage_g3(int st, const BSys *sys, int ns, const int *sel, int level, int grid, cudaStream_t s) {
  switch (st) {
    case BS_AP: return bstage_launch_t<BS_AP>(sys, ns, sel, level, grid, s);
    case BS_TRUERES: return bstage_launch_t<BS_TRUERES>(sys, ns, sel, level, grid, s);
    case BS_TUNE_A: return bstage_launch_t<BS_TUNE_A>(sys, ns, sel, level, grid, s);
    case BS_TUNE_P: return bstage_launch_t<BS_TUNE_P>(sys, ns, sel, level, grid, s);
    case BS_TUNE_R: return bstage_launch_t<BS_TUNE_R>(sys, ns, sel, level, grid, s);
    default: return -2;
  }
}

}  // namespace xamg
