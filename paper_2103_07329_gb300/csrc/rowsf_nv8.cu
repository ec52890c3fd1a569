// Fused row kernels, FP32 blocks (float or bf16 values), 8 column(s).
#define XAMG_NV 8
#define XAMG_FLOAT 1
#include "rows_inst.cuh"
