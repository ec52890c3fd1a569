// vtail_f32.cu -- the cooperative coarse-tail kernel on FP32 blocks (FP32
// values, or bf16 values of A with their row scales), one instantiation per
// block width.
#include <cuda_bf16.h>

#include <type_traits>

#include "vtail_kern.cuh"

namespace xamg {

int launch_vtail_f32(const TailProg<float> &p, int nv, int vt, cudaStream_t st) {
  if (vt == 1) {
    switch (nv) {
      case 2: return vtail_launch<float, __nv_bfloat16, 2>(p, st);
      case 4: return vtail_launch<float, __nv_bfloat16, 4>(p, st);
      case 8: return vtail_launch<float, __nv_bfloat16, 8>(p, st);
      case 16: return vtail_launch<float, __nv_bfloat16, 16>(p, st);
      case 32: return vtail_launch<float, __nv_bfloat16, 32>(p, st);
      default: return -1;
    }
  }
  switch (nv) {
    case 2: return vtail_launch<float, float, 2>(p, st);
    case 4: return vtail_launch<float, float, 4>(p, st);
    case 8: return vtail_launch<float, float, 8>(p, st);
    case 16: return vtail_launch<float, float, 16>(p, st);
    case 32: return vtail_launch<float, float, 32>(p, st);
    default: return -1;
  }
}

}  // namespace xamg
