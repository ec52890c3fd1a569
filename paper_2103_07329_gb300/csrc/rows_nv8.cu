// Fused row kernels for blocks of 8 columns.
#define XAMG_NV 8
#include "rows_inst.cuh"
