// Fused row kernels for blocks of 1 column.
#define XAMG_NV 1
#include "rows_inst.cuh"
