// Fused row kernels, FP32 blocks (float or bf16 values), 32 column(s).
#define XAMG_NV 32
#define XAMG_FLOAT 1
#include "rows_inst.cuh"
