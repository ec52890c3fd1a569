// Fused row kernels for blocks of 32 columns.
#define XAMG_NV 32
#include "rows_inst.cuh"
