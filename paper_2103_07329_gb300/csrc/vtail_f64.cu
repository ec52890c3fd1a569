// vtail_f64.cu -- the cooperative coarse-tail kernel on FP64 blocks (FP64
// values), one instantiation per block width.
#include <type_traits>

#include "vtail_kern.cuh"

namespace xamg {

int launch_vtail_f64(const TailProg<double> &p, int nv, cudaStream_t st) {
  switch (nv) {
    case 2: return vtail_launch<double, double, 2>(p, st);
    case 4: return vtail_launch<double, double, 4>(p, st);
    case 8: return vtail_launch<double, double, 8>(p, st);
    case 16: return vtail_launch<double, double, 16>(p, st);
    case 32: return vtail_launch<double, double, 32>(p, st);
    default: return -1;
  }
}

}  // namespace xamg
