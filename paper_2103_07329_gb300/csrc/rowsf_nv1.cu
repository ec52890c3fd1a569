// Fused row kernels, FP32 blocks (float or bf16 values), 1 column(s).
#define XAMG_NV 1
#define XAMG_FLOAT 1
#include "rows_inst.cuh"
