// batch_stage2.cu -- instantiations of the batched row stages (group 2);
// the groups compile in parallel.
#include <algorithm>

#include "batch_stage.cuh"

namespace xamg {

int launch_bstage_g2(int st, const BSys *sys, int ns, const int *sel, int level, int grid, cudaStream_t s) {
  switch (st) {
    case BS_PROLONG: return bstage_launch_t<BS_PROLONG>(sys, ns, sel, level, grid, s);
    case BS_POST1: return bstage_launch_t<BS_POST1>(sys, ns, sel, level, grid, s);
    case BS_POST2: return bstage_launch_t<BS_POST2>(sys, ns, sel, level, grid, s);
    case BS_POST2_DOT2: return bstage_launch_t<BS_POST2_DOT2>(sys, ns, sel, level, grid, s);
    default: return -2;
  }
}

}  // namespace xamg
