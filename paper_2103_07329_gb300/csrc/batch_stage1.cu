// batch_stage1.cu -- instantiations of the batched row stages (group 1);
// the groups compile in parallel.
#include <algorithm>

#include "batch_stage.cuh"

namespace xamg {

int launch_bstage_g1(int st, const BSys *sys, int ns, const int *sel, int level, int grid, cudaStream_t s) {
  switch (st) {
    case BS_PRE1: return bstage_launch_t<BS_PRE1>(sys, ns, sel, level, grid, s);
    case BS_PRE2: return bstage_launch_t<BS_PRE2>(sys, ns, sel, level, grid, s);
    case BS_RESTRICT: return bstage_launch_t<BS_RESTRICT>(sys, ns, sel, level, grid, s);
    case BS_RESTRICT_C: return bstage_launch_t<BS_RESTRICT_C>(sys, ns, sel, level, grid, s);
    default: return -2;
  }
}

}  // namespace xamg
